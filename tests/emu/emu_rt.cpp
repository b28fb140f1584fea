// Fiber runtime of the kernel emulator (see wt_emu.h): one ucontext fiber
// per lane, lanes of a warp interleaved at warp collectives.
#include <sys/mman.h>
#include <ucontext.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
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
ucontext_t g_main;
Lane g_lanes[32];
int g_cur = 0;
EmuDim g_bidx{0, 0, 0}, g_bdim{32, 1, 1}, g_gdim{1, 1, 1};
void (*g_kernel)(WtArgs) = nullptr;
const WtArgs *g_args = nullptr;
// collective state
int g_arrived = 0, g_gen = 0, g_kind = 0, g_done = 0;
float g_fv[32], g_fres[32];
int g_iv[32], g_ires[32], g_arg[32];
bool g_is_int = false;
std::string g_fail;

void trampoline() {
  g_kernel(*g_args);
  g_lanes[g_cur].done = true;
  g_done++;
  swapcontext(&g_lanes[g_cur].ctx, &g_main);
}

void complete() {
  for (int l = 0; l < 32; l++) {
    int src = l;
    if (g_kind == 0) src = g_arg[l] & 31;
    else if (g_kind == 1) src = l - g_arg[l] < 0 ? l : l - g_arg[l];
    else if (g_kind == 2) src = l + g_arg[l] > 31 ? l : l + g_arg[l];
    if (g_kind == 3) {  // all
      int all = 1;
      for (int m = 0; m < 32; m++) all &= g_iv[m] != 0;
      g_ires[l] = all;
    } else if (g_kind == 4) {  // syncwarp
      g_ires[l] = 0;
    } else {
      g_fres[l] = g_fv[src];
      g_ires[l] = g_iv[src];
    }
  }
}

// Posts this lane's contribution; returns once all 32 lanes have posted.
void collective(int kind) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  if (g_arrived == 0) g_kind = kind;
  else if (g_kind != kind) {
    g_fail = "lanes reached different warp collectives";
  }
  g_arrived++;
  int gen = g_gen;
  if (g_arrived == 32) {
    complete();
    g_arrived = 0;
    g_gen++;
    return;
  }
  (void)lane;
  while (g_gen == gen) {
    if (g_arrived + g_done >= 32 && g_arrived < 32) {
      g_fail = "warp collective with exited lanes";
      g_gen++;  // release, the run is failed anyway
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
  g_fv[lane] = v;
  g_arg[lane] = arg;
  collective(kind);
  return g_fres[lane];
}
int wt_emu_shfl_i(int v, int arg, int kind) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  g_iv[lane] = v;
  g_arg[lane] = arg;
  collective(kind);
  return g_ires[lane];
}
int wt_emu_all(int pred) {
  int lane = (int)(g_lanes[g_cur].tid.x & 31);
  g_iv[lane] = pred;
  collective(3);
  return g_ires[lane];
}
void wt_emu_syncwarp() { collective(4); }
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
  for (int l = 0; l < 32; l++)
    if (!g_lanes[l].stack) {
      void *p = mmap(nullptr, kStack, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
      if (p == MAP_FAILED) {
        snprintf(msg, msg_cap, "mmap failed");
        return -1;
      }
      g_lanes[l].stack = (char *)p;
    }
  g_bdim = EmuDim{(unsigned)block, 1, 1};
  g_gdim = EmuDim{(unsigned)gx, (unsigned)gy, (unsigned)gz};
  for (int bz = 0; bz < gz; bz++)
    for (int by = 0; by < gy; by++)
      for (int bx = 0; bx < gx; bx++) {
        g_bidx = EmuDim{(unsigned)bx, (unsigned)by, (unsigned)bz};
        memset(wt_emu_smem_array, 0xA5, (size_t)smem);  // poison
        for (int w = 0; w < (block + 31) / 32; w++) {
          g_arrived = 0;
          g_done = 0;
          for (int l = 0; l < 32; l++) {
            Lane &L = g_lanes[l];
            L.done = false;
            L.tid = EmuDim{(unsigned)(w * 32 + l), 0, 0};
            getcontext(&L.ctx);
            L.ctx.uc_stack.ss_sp = L.stack;
            L.ctx.uc_stack.ss_size = kStack;
            L.ctx.uc_link = nullptr;
            makecontext(&L.ctx, trampoline, 0);
          }
          while (g_done < 32) {
            for (int l = 0; l < 32; l++) {
              if (g_lanes[l].done) continue;
              g_cur = l;
              swapcontext(&g_main, &g_lanes[l].ctx);
            }
            if (!g_fail.empty()) {
              snprintf(msg, msg_cap, "%s (block %d,%d,%d warp %d)", g_fail.c_str(), bx, by, bz, w);
              return -1;
            }
          }
        }
      }
  return 0;
}
}
