// Hand-written device helpers shared by every generated group kernel.
// The text below is prepended to each generated kernel and compiled with
// NVRTC for sm_103a.  It uses only PTX instructions (cp.async.bulk.tensor,
// mbarrier, cvt) and CUDA built-ins; no CUDA headers are needed.
#include "wt_internal.hpp"

namespace wt {

const char *kDeviceSource = R"WTDEV(
typedef unsigned long long wt_u64;
typedef long long wt_i64;
typedef unsigned int wt_u32;
typedef unsigned short wt_u16;

struct __align__(64) WtTmap { wt_u64 v[16]; };
struct WtSrc { const void *ptr; int W, H, C, dtype; wt_i64 pitch, plane; };
struct WtDst { void *ptr; int W, H, C, dtype; wt_i64 pitch, plane; };
struct __align__(64) WtArgs {
  WtTmap tmap[8];  // TMA-staged sources
  WtSrc src[24];   // staged sources, then gather sources
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
  int direct;      // 1: tile = block index (no queue)
  const void *img_tab;
  int tile_h2, ty1, ty2, n_big;
};

#define WT_FULL 0xffffffffu
#define WT_ERR_TIMEOUT 1
#define WT_ERR_BOUNDS 2
#ifndef WT_WAIT_LIMIT
#define WT_WAIT_LIMIT (1 << 22)
#endif

static __device__ __forceinline__ wt_u32 wt_smem_u32(const void *p) {
  return (wt_u32)__cvta_generic_to_shared(p);
}

static __device__ __forceinline__ void wt_mbar_init(wt_u32 bar, wt_u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
static __device__ __forceinline__ void wt_fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
static __device__ __forceinline__ void wt_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// A tensor map read from global memory (batched runs keep one per image in
// a device table written before the launch): acquire it for the async proxy
// before the first bulk tensor copy that names it.
static __device__ __forceinline__ void wt_tmap_acquire(const void *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((wt_u64)map) : "memory");
}
static __device__ __forceinline__ void wt_mbar_expect_tx(wt_u32 bar, wt_u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
static __device__ __forceinline__ wt_u32 wt_mbar_try_wait(wt_u32 bar, wt_u32 parity) {
  wt_u32 ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait: returns 1 on completion, 0 (and raises the error word) if
// the limit is reached, so a lost transfer never hangs the GPU.
static __device__ __forceinline__ int wt_mbar_wait(wt_u32 bar, wt_u32 parity, int *err) {
  for (int i = 0; i < WT_WAIT_LIMIT; i++)
    if (wt_mbar_try_wait(bar, parity)) return 1;
  atomicExch(err, WT_ERR_TIMEOUT);
  return 0;
}
// 3-D tiled TMA load of one box into shared memory, completion on `bar`.
static __device__ __forceinline__ void wt_tma_load_3d(wt_u32 dst, const WtTmap *map, int x, int y,
                                                      int z, wt_u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((wt_u64)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------ conversions
static __device__ __forceinline__ float wt_h2f(wt_u16 h) {
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
}
static __device__ __forceinline__ wt_u16 wt_f2h(float f) {
  wt_u16 h;
  asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
  return h;
}
static __device__ __forceinline__ float wt_b2f(wt_u16 b) { return __uint_as_float(((wt_u32)b) << 16); }
static __device__ __forceinline__ wt_u16 wt_f2b(float f) {
  wt_u16 h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
  return h;
}

// ------------------------------------------------- vector loads (4 lanes)
static __device__ __forceinline__ void wt_ld4_f32(const void *p, float &a, float &b, float &c,
                                                  float &d) {
  float4 v = *(const float4 *)p;
  a = v.x; b = v.y; c = v.z; d = v.w;
}
static __device__ __forceinline__ void wt_ld4_f16(const void *p, float &a, float &b, float &c,
                                                  float &d) {
  uint2 v = *(const uint2 *)p;
  a = wt_h2f((wt_u16)(v.x & 0xffff)); b = wt_h2f((wt_u16)(v.x >> 16));
  c = wt_h2f((wt_u16)(v.y & 0xffff)); d = wt_h2f((wt_u16)(v.y >> 16));
}
static __device__ __forceinline__ void wt_ld4_bf16(const void *p, float &a, float &b, float &c,
                                                   float &d) {
  uint2 v = *(const uint2 *)p;
  a = __uint_as_float(v.x << 16); b = __uint_as_float(v.x & 0xffff0000u);
  c = __uint_as_float(v.y << 16); d = __uint_as_float(v.y & 0xffff0000u);
}
// ------------------------------- read-only 8-element loads (16-byte aligned)
static __device__ __forceinline__ void wt_ld8_f32(const void *p, float &a, float &b, float &c, float &d,
                                                  float &e, float &f, float &g, float &h) {
  const float4 u = __ldg((const float4 *)p), w = __ldg((const float4 *)p + 1);
  a = u.x; b = u.y; c = u.z; d = u.w; e = w.x; f = w.y; g = w.z; h = w.w;
}
static __device__ __forceinline__ void wt_ld8_f16(const void *p, float &a, float &b, float &c, float &d,
                                                  float &e, float &f, float &g, float &h) {
  const uint4 v = __ldg((const uint4 *)p);
  a = wt_h2f((wt_u16)(v.x & 0xffff)); b = wt_h2f((wt_u16)(v.x >> 16));
  c = wt_h2f((wt_u16)(v.y & 0xffff)); d = wt_h2f((wt_u16)(v.y >> 16));
  e = wt_h2f((wt_u16)(v.z & 0xffff)); f = wt_h2f((wt_u16)(v.z >> 16));
  g = wt_h2f((wt_u16)(v.w & 0xffff)); h = wt_h2f((wt_u16)(v.w >> 16));
}
static __device__ __forceinline__ void wt_ld8_bf16(const void *p, float &a, float &b, float &c, float &d,
                                                   float &e, float &f, float &g, float &h) {
  const uint4 v = __ldg((const uint4 *)p);
  a = __uint_as_float(v.x << 16); b = __uint_as_float(v.x & 0xffff0000u);
  c = __uint_as_float(v.y << 16); d = __uint_as_float(v.y & 0xffff0000u);
  e = __uint_as_float(v.z << 16); f = __uint_as_float(v.z & 0xffff0000u);
  g = __uint_as_float(v.w << 16); h = __uint_as_float(v.w & 0xffff0000u);
}
// --------------------------------------------- shared-memory row buffers
// FP32 buffer element i of n (n: the buffer's length; bounds are checked
// where the kernels are emulated on the host)
static __device__ __forceinline__ float wt_sld(const float *b, int i, int n) { (void)n; return b[i]; }
static __device__ __forceinline__ void wt_sst(float *b, int i, int n, float v) { (void)n; b[i] = v; }
// 8 stored elements from shared memory (16-byte aligned), and one
static __device__ __forceinline__ void wt_lds8_f32(const void *p, float &a, float &b, float &c, float &d,
                                                   float &e, float &f, float &g, float &h) {
  const float4 u = ((const float4 *)p)[0], w = ((const float4 *)p)[1];
  a = u.x; b = u.y; c = u.z; d = u.w; e = w.x; f = w.y; g = w.z; h = w.w;
}
static __device__ __forceinline__ void wt_lds8_f16(const void *p, float &a, float &b, float &c, float &d,
                                                   float &e, float &f, float &g, float &h) {
  const uint4 v = *(const uint4 *)p;
  a = wt_h2f((wt_u16)(v.x & 0xffff)); b = wt_h2f((wt_u16)(v.x >> 16));
  c = wt_h2f((wt_u16)(v.y & 0xffff)); d = wt_h2f((wt_u16)(v.y >> 16));
  e = wt_h2f((wt_u16)(v.z & 0xffff)); f = wt_h2f((wt_u16)(v.z >> 16));
  g = wt_h2f((wt_u16)(v.w & 0xffff)); h = wt_h2f((wt_u16)(v.w >> 16));
}
static __device__ __forceinline__ void wt_lds8_bf16(const void *p, float &a, float &b, float &c, float &d,
                                                    float &e, float &f, float &g, float &h) {
  const uint4 v = *(const uint4 *)p;
  a = __uint_as_float(v.x << 16); b = __uint_as_float(v.x & 0xffff0000u);
  c = __uint_as_float(v.y << 16); d = __uint_as_float(v.y & 0xffff0000u);
  e = __uint_as_float(v.z << 16); f = __uint_as_float(v.z & 0xffff0000u);
  g = __uint_as_float(v.w << 16); h = __uint_as_float(v.w & 0xffff0000u);
}
static __device__ __forceinline__ float wt_lds1_f32(const void *p) { return *(const float *)p; }
static __device__ __forceinline__ float wt_lds1_f16(const void *p) { return wt_h2f(*(const wt_u16 *)p); }
static __device__ __forceinline__ float wt_lds1_bf16(const void *p) { return wt_b2f(*(const wt_u16 *)p); }
// ------------------------------------- asynchronous copies global -> shared
// 16 bytes (both addresses 16-byte aligned); completion by commit groups
static __device__ __forceinline__ void wt_cp_async16(wt_u32 dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// 4 bytes (both addresses 4-byte aligned)
static __device__ __forceinline__ void wt_cp_async4(wt_u32 dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
// the 16-byte copy only where p holds (predicated, no branch)
static __device__ __forceinline__ void wt_cp_async16_if(bool p, wt_u32 dst, const void *src) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q cp.async.cg.shared.global [%1], [%2], 16;\n}" ::"r"((int)p),
               "r"(dst), "l"(src)
               : "memory");
}
static __device__ __forceinline__ void wt_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
#define WT_CP_ASYNC_WAIT(n) asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory")
// ------------------------------- read-only pairs (aligned to their size)
static __device__ __forceinline__ void wt_ld2_f32(const void *p, float &a, float &b) {
  const float2 v = __ldg((const float2 *)p);
  a = v.x; b = v.y;
}
static __device__ __forceinline__ void wt_ld2_f16(const void *p, float &a, float &b) {
  const wt_u32 v = __ldg((const unsigned int *)p);
  a = wt_h2f((wt_u16)(v & 0xffff)); b = wt_h2f((wt_u16)(v >> 16));
}
static __device__ __forceinline__ void wt_ld2_bf16(const void *p, float &a, float &b) {
  const wt_u32 v = __ldg((const unsigned int *)p);
  a = __uint_as_float(v << 16); b = __uint_as_float(v & 0xffff0000u);
}
// ------------------------------------------------ vector stores (4 lanes)
static __device__ __forceinline__ void wt_st4_f32(void *p, float a, float b, float c, float d) {
  *(float4 *)p = make_float4(a, b, c, d);
}
// two values rounded (RNE) and packed in one conversion: lo in bits 0-15,
// hi in bits 16-31 (the instruction puts its first source in the upper half)
static __device__ __forceinline__ wt_u32 wt_f2h2(float lo, float hi) {
  wt_u32 r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
static __device__ __forceinline__ wt_u32 wt_f2b2(float lo, float hi) {
  wt_u32 r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
static __device__ __forceinline__ void wt_st4_f16(void *p, float a, float b, float c, float d) {
  *(uint2 *)p = make_uint2(wt_f2h2(a, b), wt_f2h2(c, d));
}
static __device__ __forceinline__ void wt_st4_bf16(void *p, float a, float b, float c, float d) {
  *(uint2 *)p = make_uint2(wt_f2b2(a, b), wt_f2b2(c, d));
}
// ------------------------------------------------------- scalar accesses
static __device__ __forceinline__ float wt_ld1_f32(const void *p) { return __ldg((const float *)p); }
static __device__ __forceinline__ float wt_ld1_f16(const void *p) {
  return wt_h2f(__ldg((const unsigned short *)p));
}
static __device__ __forceinline__ float wt_ld1_bf16(const void *p) {
  return wt_b2f(__ldg((const unsigned short *)p));
}
static __device__ __forceinline__ void wt_st1_f32(void *p, float v) { *(float *)p = v; }
static __device__ __forceinline__ void wt_st1_f16(void *p, float v) { *(wt_u16 *)p = wt_f2h(v); }
static __device__ __forceinline__ void wt_st1_bf16(void *p, float v) { *(wt_u16 *)p = wt_f2b(v); }

static __device__ __forceinline__ int wt_clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}
// ---------------------------------------- packed FP32 pairs (sm_100+)
// Two FP32 lanes per instruction; each lane rounds like the scalar op.
static __device__ __forceinline__ wt_u64 wt_pk(float a, float b) {
  wt_u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
static __device__ __forceinline__ void wt_upk(wt_u64 v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
static __device__ __forceinline__ wt_u64 wt_add2(wt_u64 a, wt_u64 b) {
  wt_u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
static __device__ __forceinline__ wt_u64 wt_sub2(wt_u64 a, wt_u64 b) {
  wt_u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
static __device__ __forceinline__ wt_u64 wt_mul2(wt_u64 a, wt_u64 b) {
  wt_u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
static __device__ __forceinline__ wt_u64 wt_fma2(wt_u64 a, wt_u64 b, wt_u64 c) {
  wt_u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
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
// WT-DEVICE-HELPERS-END
)WTDEV";

}  // namespace wt
