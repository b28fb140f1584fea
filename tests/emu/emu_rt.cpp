// Fiber runtime of the kernel emulator (see wt_emu.h): one ucontext fiber
// per thread of a block; lanes of a warp meet at warp collectives, all
// threads of the block at block barriers.
#include <sys/mman.h>
#include <ucontext.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "wt_emu.h"

alignas(128) unsigned char wt_emu_smem_array[232 * 1024];

namespace {
constexpr size_t kStack = 4u << 20;
struct Lane {
  ucontext_t ctx;
  char *stack = nullptr;
  bool done = false;
  EmuDim tid{0, 0, 0};
};
// Per warp: the state of the warp collective in progress.
struct Warp {
  int arrived = 0, gen = 0, kind = 0, done = 0, size = 32;
  float fv[32], fres[32];
  int iv[32], ires[32], arg[32];
};
ucontext_t g_main;
std::vector<Lane> g_lanes;  // every thread of the block being run
std::vector<Warp> g_warps;
int g_cur = 0;
int g_block_threads = 0, g_block_done = 0, g_bar_arrived = 0, g_bar_gen = 0;
EmuDim g_bidx{0, 0, 0}, g_bdim{32, 1, 1}, g_gdim{1, 1, 1};
void (*g_kernel)(WtArgs) = nullptr;
const WtArgs *g_args = nullptr;
std::string g_fail;

void trampoline() {
  g_kernel(*g_args);
  Lane &L = g_lanes[g_cur];
  L.done = true;
  g_warps[L.tid.x / 32].done++;
  g_block_done++;
  swapcontext(&L.ctx, &g_main);
}

void complete(Warp &W) {
  for (int l = 0; l < W.size; l++) {
    int src = l;
    if (W.kind == 0) src = W.arg[l] & 31;
    else if (W.kind == 1) src = l - W.arg[l] < 0 ? l : l - W.arg[l];
    else if (W.kind == 2) src = l + W.arg[l] > 31 ? l : l + W.arg[l];
    if (src >= W.size) src = l;
    if (W.kind == 3) {  // all
      int all = 1;
      for (int m = 0; m < W.size; m++) all &= W.iv[m] != 0;
      W.ires[l] = all;
    } else if (W.kind == 4) {  // syncwarp
      W.ires[l] = 0;
    } else {
      W.fres[l] = W.fv[src];
      W.ires[l] = W.iv[src];
    }
  }
}

Warp &my_warp() { return g_warps[g_lanes[g_cur].tid.x / 32]; }

// Posts this lane's contribution; returns once every lane of its warp has.
void collective(int kind) {
  Warp &W = my_warp();
  if (W.arrived == 0) W.kind = kind;
  else if (W.kind != kind) g_fail = "lanes reached different warp collectives";
  W.arrived++;
  int gen = W.gen;
  if (W.arrived == W.size) {
    complete(W);
    W.arrived = 0;
    W.gen++;
    return;
  }
  while (W.gen == gen) {
    if (W.arrived + W.done >= W.size && W.arrived < W.size) {
      g_fail = "warp collective with exited lanes";
      W.gen++;  // release, the run is failed anyway
      break;
    }
    swapcontext(&g_lanes[g_cur].ctx, &g_main);
  }
}

// Block-wide barrier: returns once every thread of the block has arrived.
void block_barrier() {
  g_bar_arrived++;
  int gen = g_bar_gen;
  if (g_bar_arrived == g_block_threads) {
    g_bar_arrived = 0;
    g_bar_gen++;
    return;
  }
  while (g_bar_gen == gen) {
    if (g_bar_arrived + g_block_done >= g_block_threads && g_bar_arrived < g_block_threads) {
      g_fail = "block barrier with exited threads";
      g_bar_gen++;
      break;
    }
    swapcontext(&g_lanes[g_cur].ctx, &g_main);
  }
}
}  // namespace

extern "C" {
EmuDim *wt_emu_thread_idx() { return &g_lanes[g_cur].tid; }
EmuDim *wt_emu_block_idx() { return &g_bidx; }
EmuDim *wt_emu_block_dim() { return &g_bdim; }
EmuDim *wt_emu_grid_dim() { return &g_gdim; }
unsigned char *wt_emu_smem() { return wt_emu_smem_array; }
void wt_emu_fail(const char *msg) {
  if (g_fail.empty()) g_fail = msg;
}

// Memory checker: every access of the generated code's load/store helpers
// must fall inside the launch's shared-memory size or a registered global
// buffer (the images of the run).
static std::vector<std::pair<const unsigned char *, size_t>> g_ranges;
static size_t g_smem_size = 0;
void wt_emu_register(const void *p, long bytes) { g_ranges.push_back({(const unsigned char *)p, (size_t)bytes}); }
void wt_emu_clear_ranges() { g_ranges.clear(); }
long wt_emu_smem_size() { return (long)g_smem_size; }
bool wt_emu_in_global(const void *p, long bytes) {
  const unsigned char *a = (const unsigned char *)p;
  for (auto &r : g_ranges)
    if (a >= r.first && a + bytes <= r.first + r.second) return true;
  return false;
}

void wt_emu_check(const void *p, long bytes, const char *what) {
  const unsigned char *a = (const unsigned char *)p;
  if (a >= wt_emu_smem_array && a + bytes <= wt_emu_smem_array + g_smem_size) return;
  for (auto &r : g_ranges)
    if (a >= r.first && a + bytes <= r.first + r.second) return;
  char m[160];
  snprintf(m, sizeof m, "out-of-bounds %s of %ld bytes (shared offset %ld)", what, bytes,
           (long)(a - wt_emu_smem_array));
  wt_emu_fail(m);
}

float wt_emu_shfl(float v, int arg, int kind) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  Warp &W = my_warp();
  W.fv[lane] = v;
  W.arg[lane] = arg;
  collective(kind);
  return W.fres[lane];
}
int wt_emu_shfl_i(int v, int arg, int kind) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  Warp &W = my_warp();
  W.iv[lane] = v;
  W.arg[lane] = arg;
  collective(kind);
  return W.ires[lane];
}
int wt_emu_all(int pred) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  Warp &W = my_warp();
  W.iv[lane] = pred;
  collective(3);
  return W.ires[lane];
}
void wt_emu_syncwarp() { collective(4); }
void wt_emu_syncthreads() { block_barrier(); }
void wt_emu_yield() { swapcontext(&g_lanes[g_cur].ctx, &g_main); }

// Runs the whole grid, one warp at a time.  Returns 0, or -1 with a message.
int wt_emu_run(void *kernel, const void *args, int gx, int gy, int gz, int block, int smem, char *msg,
               int msg_cap) {
  g_smem_size = (size_t)smem;
  g_kernel = (void (*)(WtArgs))kernel;
  g_args = (const WtArgs *)args;
  g_fail.clear();
  if (smem > (int)sizeof(wt_emu_smem_array)) {
    snprintf(msg, msg_cap, "shared memory request too large");
    return -1;
  }
  if (block < 1 || block > 1024) {
    snprintf(msg, msg_cap, "bad block size");
    return -1;
  }
  if ((int)g_lanes.size() < block) g_lanes.resize(block);
  for (int l = 0; l < block; l++)
    if (!g_lanes[l].stack) {
      void *p = mmap(nullptr, kStack, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE, -1, 0);
      if (p == MAP_FAILED) {
        snprintf(msg, msg_cap, "mmap failed");
        return -1;
      }
      g_lanes[l].stack = (char *)p;
    }
  g_bdim = EmuDim{(unsigned)block, 1, 1};
  g_gdim = EmuDim{(unsigned)gx, (unsigned)gy, (unsigned)gz};
  const int nwarps = (block + 31) / 32;
  for (int bz = 0; bz < gz; bz++)
    for (int by = 0; by < gy; by++)
      for (int bx = 0; bx < gx; bx++) {
        g_bidx = EmuDim{(unsigned)bx, (unsigned)by, (unsigned)bz};
        memset(wt_emu_smem_array, 0xA5, (size_t)smem);  // poison
        // every thread of the block is a fiber: warps interleave at warp
        // collectives and block barriers
        g_warps.assign(nwarps, Warp());
        for (int w = 0; w < nwarps; w++) g_warps[w].size = std::min(32, block - 32 * w);
        g_block_threads = block;
        g_block_done = 0;
        g_bar_arrived = 0;
        for (int l = 0; l < block; l++) {
          Lane &L = g_lanes[l];
          L.done = false;
          L.tid = EmuDim{(unsigned)l, 0, 0};
          getcontext(&L.ctx);
          L.ctx.uc_stack.ss_sp = L.stack;
          L.ctx.uc_stack.ss_size = kStack;
          L.ctx.uc_link = nullptr;
          makecontext(&L.ctx, trampoline, 0);
        }
        while (g_block_done < block) {
          for (int l = 0; l < block; l++) {
            if (g_lanes[l].done) continue;
            g_cur = l;
            swapcontext(&g_main, &g_lanes[l].ctx);
          }
          if (!g_fail.empty()) {
            snprintf(msg, msg_cap, "%s (block %d,%d,%d)", g_fail.c_str(), bx, by, bz);
            return -1;
          }
        }
      }
  return 0;
}
}
