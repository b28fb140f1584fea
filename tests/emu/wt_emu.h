// Host emulation of the device helpers used by generated group kernels.
//
// Test infrastructure for the CUDA path: the kernel text that the library
// generates (everything after its device-helper block) is compiled as host
// C++ against this header and run with one cooperative fiber per lane, so
// the tiling, halo, clamping and load-type logic can be checked against the
// oracle on a machine without a GPU.  Warp collectives (__shfl_*_sync,
// __all_sync, __syncwarp) are exchanges among the 32 fibers of a warp; TMA
// copies complete synchronously; mbarriers track phases.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <algorithm>

typedef unsigned long long wt_u64;
typedef long long wt_i64;
typedef unsigned int wt_u32;
typedef unsigned short wt_u16;

#define __global__
#define __device__
#define __forceinline__ inline
#define __grid_constant__
#define __launch_bounds__(...)
#define __shared__
#define __align__(n) __attribute__((aligned(n)))

struct alignas(64) WtTmap { wt_u64 v[16]; };
struct WtSrc { const void *ptr; int W, H, C, dtype; wt_i64 pitch, plane; };
struct WtDst { void *ptr; int W, H, C, dtype; wt_i64 pitch, plane; };
struct alignas(64) WtArgs {
  WtTmap tmap[8];
  WtSrc src[24];
  WtDst dst[8];
  int W, H;
  int tile_h, tiles_x, tiles_y, n_tiles;
  int chunk, nbuf;
  int out_w;
  int channels;
  int *err;
  const int *tile_table;
  int *queue;
  int n_images;
  int direct;
  const void *img_tab;
  int tile_h2, ty1, ty2, n_big;
};
struct EmuTmap {  // the library's debug encoding of a tensor-map slot
  const void *ptr;
  int32_t W, H, C, esz;
  int64_t pitch, plane;
  int32_t boxw, boxh;
};

struct float4 { float x, y, z, w; };
struct uint2 { unsigned x, y; };
static inline float4 make_float4(float a, float b, float c, float d) { return float4{a, b, c, d}; }
struct EmuDim { unsigned x, y, z; };

#define WT_FULL 0xffffffffu
#define WT_ERR_TIMEOUT 1
#define WT_ERR_BOUNDS 2

// ---------------------------------------------------------- fiber runtime
extern "C" {
EmuDim *wt_emu_thread_idx();
EmuDim *wt_emu_block_idx();
EmuDim *wt_emu_block_dim();
EmuDim *wt_emu_grid_dim();
float wt_emu_shfl(float v, int src_lane, int kind);  // kind 0 idx, 1 up, 2 down
int wt_emu_shfl_i(int v, int src_lane, int kind);
int wt_emu_all(int pred);
void wt_emu_syncwarp();
void wt_emu_syncthreads();
unsigned char *wt_emu_smem();
long wt_emu_smem_size();
bool wt_emu_in_global(const void *p, long bytes);
void wt_emu_fail(const char *msg);
void wt_emu_check(const void *p, long bytes, const char *what);
void wt_emu_yield();
}
#define threadIdx (*wt_emu_thread_idx())
#define blockIdx (*wt_emu_block_idx())
#define blockDim (*wt_emu_block_dim())
#define gridDim (*wt_emu_grid_dim())
#define wt_smem wt_emu_smem_array

static inline float __shfl_sync(unsigned, float v, int l) { return wt_emu_shfl(v, l, 0); }
static inline int __shfl_sync(unsigned, int v, int l) { return wt_emu_shfl_i(v, l, 0); }
static inline float __shfl_up_sync(unsigned, float v, int d) { return wt_emu_shfl(v, d, 1); }
static inline float __shfl_down_sync(unsigned, float v, int d) { return wt_emu_shfl(v, d, 2); }
static inline int __all_sync(unsigned, int p) { return wt_emu_all(p); }
static inline void __syncwarp(unsigned = 0xffffffffu) { wt_emu_syncwarp(); }
static inline void __syncthreads() { wt_emu_syncthreads(); }
static inline int atomicAdd(int *p, int v) { int o = *p; *p += v; return o; }
static inline int atomicExch(int *p, int v) { int o = *p; *p = v; return o; }
static inline void __threadfence() {}
using std::min;
using std::max;

static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline float __int_as_float(int u) { float f; memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }

// ------------------------------------------------------ shared memory
static inline wt_u32 wt_smem_u32(const void *p) {
  return (wt_u32)((const unsigned char *)p - wt_emu_smem());
}
static inline unsigned char *wt_emu_sptr(wt_u32 a) { return wt_emu_smem() + a; }

// ------------------------------------------------------ mbarrier / TMA
// An emulated mbarrier keeps its completed-phase count in the first 4 bytes
// and the transaction bytes still expected in the current phase in the next
// 4 (arrival count 1: one arrive.expect_tx per phase).  A phase completes
// when its arrival has happened and every expected byte has been copied, so
// a phase armed for bytes that no copy delivers never completes.
static inline void wt_mbar_init(wt_u32 bar, wt_u32) {
  wt_emu_check(wt_emu_sptr(bar), 8, "mbarrier");
  memset(wt_emu_sptr(bar), 0, 8);
}
static inline void wt_fence_mbar_init() {}
static inline void wt_fence_proxy_async() {}
static inline void wt_tmap_acquire(const void *) {}
static inline void wt_emu_mbar_tx(wt_u32 bar, int32_t delta) {
  int32_t ph, tx;
  memcpy(&ph, wt_emu_sptr(bar), 4);
  memcpy(&tx, wt_emu_sptr(bar) + 4, 4);
  tx += delta;
  if (tx < 0) wt_emu_fail("mbarrier: more bytes copied than expected");
  if (tx == 0) ph++;
  memcpy(wt_emu_sptr(bar), &ph, 4);
  memcpy(wt_emu_sptr(bar) + 4, &tx, 4);
}
static inline void wt_mbar_expect_tx(wt_u32 bar, wt_u32 bytes) {
  int32_t tx;
  memcpy(&tx, wt_emu_sptr(bar) + 4, 4);
  if (tx != 0) wt_emu_fail("mbarrier armed again before its phase completed");
  wt_emu_mbar_tx(bar, (int32_t)bytes);
}
static inline wt_u32 wt_mbar_try_wait(wt_u32 bar, wt_u32 parity) {
  int32_t ph;
  memcpy(&ph, wt_emu_sptr(bar), 4);
  // phase `parity` is complete when the count of completed phases has the
  // other parity and at least one phase completed since it began
  return (wt_u32)(ph > 0 && (((wt_u32)ph - 1) & 1u) == parity);
}
static inline int wt_mbar_wait(wt_u32 bar, wt_u32 parity, int *err) {
  // another lane of the warp may still have to issue the copy: yield
  for (int i = 0; i < 64; i++) {
    if (wt_mbar_try_wait(bar, parity)) return 1;
    wt_emu_yield();
  }
  atomicExch(err, WT_ERR_TIMEOUT);
  return 0;
}
static inline void wt_tma_load_3d(wt_u32 dst, const WtTmap *map, int x, int y, int z, wt_u32 bar) {
  EmuTmap t;
  memcpy(&t, map, sizeof t);
  unsigned char *d = wt_emu_sptr(dst);
  wt_emu_check(d, (long)t.boxw * t.boxh * t.esz, "TMA box");
  wt_emu_check(wt_emu_sptr(bar), 8, "mbarrier");
  if (dst % 128 != 0) wt_emu_fail("TMA destination not 128-byte aligned");
  if (((long)x * t.esz) % 16 != 0) wt_emu_fail("TMA x coordinate not 16-byte aligned");
  for (int r = 0; r < t.boxh; r++)
    for (int c = 0; c < t.boxw; c++) {
      int gx = x + c, gy = y + r;
      unsigned char *o = d + ((size_t)r * t.boxw + c) * t.esz;
      if (gx < 0 || gx >= t.W || gy < 0 || gy >= t.H || z < 0 || z >= t.C) {
        memset(o, 0, t.esz);
      } else {
        const unsigned char *s = (const unsigned char *)t.ptr + (int64_t)z * t.plane + (int64_t)gy * t.pitch +
                                 (int64_t)gx * t.esz;
        memcpy(o, s, t.esz);
      }
    }
  // the whole box counts towards the barrier's transaction bytes
  wt_emu_mbar_tx(bar, -(int32_t)((long)t.boxw * t.boxh * t.esz));
}

// ------------------------------------------------------ conversions
static inline float wt_h2f(wt_u16 h) {
  unsigned s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  float v;
  if (e == 0) v = std::ldexp((float)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp((float)(m | 1024), (int)e - 25);
  return s ? -v : v;
}
static inline wt_u16 wt_f2h(float f) {  // round to nearest even
  unsigned x = __float_as_uint(f), sign = (x >> 16) & 0x8000u, ax = x & 0x7fffffffu;
  if (ax >= 0x7f800000u) return (wt_u16)(sign | (ax > 0x7f800000u ? 0x7e00u : 0x7c00u));
  if (ax >= 0x477ff000u) return (wt_u16)(sign | 0x7c00u);
  if (ax < 0x38800000u) {
    double r = std::nearbyint((double)__uint_as_float(ax) * 16777216.0);
    return (wt_u16)(sign | (unsigned)r);
  }
  unsigned m = ax + 0x0fffu + ((ax >> 13) & 1u);
  m -= 0x38000000u;
  return (wt_u16)(sign | (m >> 13));
}
static inline float wt_b2f(wt_u16 b) { return __uint_as_float(((wt_u32)b) << 16); }
static inline wt_u16 wt_f2b(float f) {
  unsigned u = __float_as_uint(f);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (wt_u16)((u >> 16) | 0x40u);
  return (wt_u16)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

// ------------------------------------------------------ loads / stores
// vector accesses must be naturally aligned, as on the GPU
static inline void wt_emu_align(const void *p, long bytes) {
  if ((long)((unsigned long)p % (unsigned long)bytes) != 0) wt_emu_fail("misaligned vector access");
}
static inline void wt_ld8_f32(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                              float &g, float &h) {
  wt_emu_check(p, 32, "load");
  wt_emu_align(p, 16);
  float v[8];
  memcpy(v, p, 32);
  a = v[0]; b = v[1]; c = v[2]; d = v[3]; e = v[4]; f = v[5]; g = v[6]; h = v[7];
}
static inline void wt_ld8_f16(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                              float &g, float &h) {
  wt_emu_check(p, 16, "load");
  wt_emu_align(p, 16);
  wt_u16 v[8];
  memcpy(v, p, 16);
  a = wt_h2f(v[0]); b = wt_h2f(v[1]); c = wt_h2f(v[2]); d = wt_h2f(v[3]);
  e = wt_h2f(v[4]); f = wt_h2f(v[5]); g = wt_h2f(v[6]); h = wt_h2f(v[7]);
}
static inline void wt_ld8_bf16(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                               float &g, float &h) {
  wt_emu_check(p, 16, "load");
  wt_emu_align(p, 16);
  wt_u16 v[8];
  memcpy(v, p, 16);
  a = wt_b2f(v[0]); b = wt_b2f(v[1]); c = wt_b2f(v[2]); d = wt_b2f(v[3]);
  e = wt_b2f(v[4]); f = wt_b2f(v[5]); g = wt_b2f(v[6]); h = wt_b2f(v[7]);
}
static inline bool wt_emu_in_smem(const void *p, long bytes) {
  const unsigned char *a = (const unsigned char *)p;
  return a >= wt_emu_smem() && a + bytes <= wt_emu_smem() + wt_emu_smem_size();
}
static inline float wt_sld(const float *b, int i, int n) {
  if (i < 0 || i >= n || !wt_emu_in_smem(b + i, 4)) {
    wt_emu_fail("shared buffer index out of range (load)");
    return 0.f;
  }
  return b[i];
}
static inline void wt_sst(float *b, int i, int n, float v) {
  if (i < 0 || i >= n || !wt_emu_in_smem(b + i, 4)) {
    wt_emu_fail("shared buffer index out of range (store)");
    return;
  }
  b[i] = v;
}
static inline void wt_lds8_f32(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                               float &g, float &h) {
  if (!wt_emu_in_smem(p, 32) || ((unsigned long)p) % 16 != 0) {
    wt_emu_fail("shared 32-byte load outside shared memory or misaligned");
    a = b = c = d = e = f = g = h = 0.f;
    return;
  }
  wt_ld8_f32(p, a, b, c, d, e, f, g, h);
}
static inline void wt_lds8_f16(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                               float &g, float &h) {
  if (!wt_emu_in_smem(p, 16) || ((unsigned long)p) % 16 != 0) {
    wt_emu_fail("shared 16-byte load outside shared memory or misaligned");
    a = b = c = d = e = f = g = h = 0.f;
    return;
  }
  wt_ld8_f16(p, a, b, c, d, e, f, g, h);
}
static inline void wt_lds8_bf16(const void *p, float &a, float &b, float &c, float &d, float &e, float &f,
                                float &g, float &h) {
  if (!wt_emu_in_smem(p, 16) || ((unsigned long)p) % 16 != 0) {
    wt_emu_fail("shared 16-byte load outside shared memory or misaligned");
    a = b = c = d = e = f = g = h = 0.f;
    return;
  }
  wt_ld8_bf16(p, a, b, c, d, e, f, g, h);
}
static inline float wt_lds1_f32(const void *p) {
  if (!wt_emu_in_smem(p, 4)) { wt_emu_fail("shared load outside shared memory"); return 0.f; }
  float v; memcpy(&v, p, 4); return v;
}
static inline float wt_lds1_f16(const void *p) {
  if (!wt_emu_in_smem(p, 2)) { wt_emu_fail("shared load outside shared memory"); return 0.f; }
  wt_u16 v; memcpy(&v, p, 2); return wt_h2f(v);
}
static inline float wt_lds1_bf16(const void *p) {
  if (!wt_emu_in_smem(p, 2)) { wt_emu_fail("shared load outside shared memory"); return 0.f; }
  wt_u16 v; memcpy(&v, p, 2); return wt_b2f(v);
}
// cp.async: the copy completes at issue (a valid completion order); the
// source must lie in a registered global buffer, the destination in shared
// memory, both 16-byte aligned
static inline void wt_cp_async16(wt_u32 dst, const void *src) {
  if (dst % 16 != 0 || ((unsigned long)src) % 16 != 0) { wt_emu_fail("cp.async address not 16-byte aligned"); return; }
  if (!wt_emu_in_smem(wt_emu_sptr(dst), 16)) { wt_emu_fail("cp.async destination outside shared memory"); return; }
  if (wt_emu_in_smem(src, 16)) { wt_emu_fail("cp.async source in shared memory"); return; }
  if (!wt_emu_in_global(src, 16)) { wt_emu_fail("cp.async source outside the registered buffers"); return; }
  memcpy(wt_emu_sptr(dst), src, 16);
}
static inline void wt_cp_async4(wt_u32 dst, const void *src) {
  if (dst % 4 != 0 || ((unsigned long)src) % 4 != 0) { wt_emu_fail("cp.async address not 4-byte aligned"); return; }
  if (!wt_emu_in_smem(wt_emu_sptr(dst), 4)) { wt_emu_fail("cp.async destination outside shared memory"); return; }
  if (wt_emu_in_smem(src, 4)) { wt_emu_fail("cp.async source in shared memory"); return; }
  if (!wt_emu_in_global(src, 4)) { wt_emu_fail("cp.async source outside the registered buffers"); return; }
  memcpy(wt_emu_sptr(dst), src, 4);
}
static inline void wt_cp_async16_if(bool p, wt_u32 dst, const void *src) {
  if (p) wt_cp_async16(dst, src);
}
static inline void wt_cp_async_commit() {}
#define WT_CP_ASYNC_WAIT(n) ((void)(n))
static inline void wt_ld2_f32(const void *p, float &a, float &b) {
  wt_emu_check(p, 8, "load");
  wt_emu_align(p, 8);
  float v[2];
  memcpy(v, p, 8);
  a = v[0]; b = v[1];
}
static inline void wt_ld2_f16(const void *p, float &a, float &b) {
  wt_emu_check(p, 4, "load");
  wt_emu_align(p, 4);
  wt_u16 v[2];
  memcpy(v, p, 4);
  a = wt_h2f(v[0]); b = wt_h2f(v[1]);
}
static inline void wt_ld2_bf16(const void *p, float &a, float &b) {
  wt_emu_check(p, 4, "load");
  wt_emu_align(p, 4);
  wt_u16 v[2];
  memcpy(v, p, 4);
  a = wt_b2f(v[0]); b = wt_b2f(v[1]);
}
static inline void wt_ld4_f32(const void *p, float &a, float &b, float &c, float &d) {
  wt_emu_check(p, 16, "load");
  wt_emu_align(p, 16);
  float v[4];
  memcpy(v, p, 16);
  a = v[0]; b = v[1]; c = v[2]; d = v[3];
}
static inline void wt_ld4_f16(const void *p, float &a, float &b, float &c, float &d) {
  wt_emu_check(p, 8, "load");
  wt_emu_align(p, 8);
  wt_u16 v[4];
  memcpy(v, p, 8);
  a = wt_h2f(v[0]); b = wt_h2f(v[1]); c = wt_h2f(v[2]); d = wt_h2f(v[3]);
}
static inline void wt_ld4_bf16(const void *p, float &a, float &b, float &c, float &d) {
  wt_emu_check(p, 8, "load");
  wt_emu_align(p, 8);
  wt_u16 v[4];
  memcpy(v, p, 8);
  a = wt_b2f(v[0]); b = wt_b2f(v[1]); c = wt_b2f(v[2]); d = wt_b2f(v[3]);
}
static inline void wt_st4_f32(void *p, float a, float b, float c, float d) {
  wt_emu_check(p, 16, "store");
  wt_emu_align(p, 16);
  float v[4] = {a, b, c, d};
  memcpy(p, v, 16);
}
static inline void wt_st4_f16(void *p, float a, float b, float c, float d) {
  wt_emu_check(p, 8, "store");
  wt_emu_align(p, 8);
  wt_u16 v[4] = {wt_f2h(a), wt_f2h(b), wt_f2h(c), wt_f2h(d)};
  memcpy(p, v, 8);
}
static inline void wt_st4_bf16(void *p, float a, float b, float c, float d) {
  wt_emu_check(p, 8, "store");
  wt_emu_align(p, 8);
  wt_u16 v[4] = {wt_f2b(a), wt_f2b(b), wt_f2b(c), wt_f2b(d)};
  memcpy(p, v, 8);
}
static inline float wt_ld1_f32(const void *p) { wt_emu_check(p, 4, "load"); float v; memcpy(&v, p, 4); return v; }
static inline float wt_ld1_f16(const void *p) { wt_emu_check(p, 2, "load"); wt_u16 v; memcpy(&v, p, 2); return wt_h2f(v); }
static inline float wt_ld1_bf16(const void *p) { wt_emu_check(p, 2, "load"); wt_u16 v; memcpy(&v, p, 2); return wt_b2f(v); }
static inline void wt_st1_f32(void *p, float v) { wt_emu_check(p, 4, "store"); memcpy(p, &v, 4); }
static inline void wt_st1_f16(void *p, float v) { wt_emu_check(p, 2, "store"); wt_u16 h = wt_f2h(v); memcpy(p, &h, 2); }
static inline void wt_st1_bf16(void *p, float v) { wt_emu_check(p, 2, "store"); wt_u16 h = wt_f2b(v); memcpy(p, &h, 2); }
static inline int wt_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------- packed FP32 pairs
static inline wt_u64 wt_pk(float a, float b) {
  wt_u64 r;
  unsigned ua = __float_as_uint(a), ub = __float_as_uint(b);
  r = (wt_u64)ua | ((wt_u64)ub << 32);
  return r;
}
static inline void wt_upk(wt_u64 v, float &a, float &b) {
  a = __uint_as_float((unsigned)(v & 0xffffffffu));
  b = __uint_as_float((unsigned)(v >> 32));
}
static inline wt_u64 wt_add2(wt_u64 x, wt_u64 y) {
  float a, b, c, d; wt_upk(x, a, b); wt_upk(y, c, d); return wt_pk(a + c, b + d);
}
static inline wt_u64 wt_sub2(wt_u64 x, wt_u64 y) {
  float a, b, c, d; wt_upk(x, a, b); wt_upk(y, c, d); return wt_pk(a - c, b - d);
}
static inline wt_u64 wt_mul2(wt_u64 x, wt_u64 y) {
  float a, b, c, d; wt_upk(x, a, b); wt_upk(y, c, d); return wt_pk(a * c, b * d);
}
static inline wt_u64 wt_fma2(wt_u64 x, wt_u64 y, wt_u64 z) {
  float a, b, c, d, e, f; wt_upk(x, a, b); wt_upk(y, c, d); wt_upk(z, e, f);
  return wt_pk(std::fma(a, c, e), std::fma(b, d, f));
}

// Gather-source tap: the pixel (x, y) of channel c, clamped to the
// source's domain (clamp-to-edge), through the read-only path.
#define WT_GATHER(T, ESZ)                                                                  \
  static __device__ __forceinline__ float wt_gather_##T(const WtSrc &s, int c, int x, int y) { \
    x = wt_clampi(x, 0, s.W - 1);                                                          \
    y = wt_clampi(y, 0, s.H - 1);                                                          \
    return wt_ld1_##T((const unsigned char *)s.ptr + (wt_i64)c * s.plane + (wt_i64)y * s.pitch + \
                      (wt_i64)x * ESZ);                                                   \
  }
WT_GATHER(f32, 4)
WT_GATHER(f16, 2)
WT_GATHER(bf16, 2)
#undef WT_GATHER
