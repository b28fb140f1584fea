// Batched runtime: n independent images of any sizes, one persistent launch
// per schedule group.
//
// Every group kernel of a batch is the persistent variant of the group's
// fused kernel: its warps pull tiles from one device queue that spans all
// images, and each tile names its image, so a batch of uneven images costs
// one launch per group instead of one per image and group, and the tail of
// one image overlaps the start of the next (the idle-block term `extraTBs`
// of Alg. 2 is paid once per batch).  Per image the kernel reads an argument
// block (tensor maps, output descriptors, sizes) from a device table; tiles
// are listed in a device table of (image, tile column, tile row, channel).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "wt_jit.hpp"
#include "wt_runtime.hpp"
#include "wt_sched.hpp"

namespace wt {

struct BatchCache {
  int device = -1;
  uint64_t sched_version = 0, ws_generation = 0;
  std::string key;            // raw bytes of the image descriptors
  void *table = nullptr;      // device: per launch, argument blocks then tiles
  int64_t table_bytes = 0;
  CachedRun run;
  ~BatchCache() {
    dev_free(table, (size_t)table_bytes);
  }
};

namespace {

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

}  // namespace

BatchPlan build_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n) {
  const int n_in = (int)p.in_channels.size(), n_out = (int)p.outputs.size();
  if (n < 1) fail(WT_EINVAL, "a batch needs at least one image");
  BatchPlan b;
  b.img.reserve(n);
  for (int i = 0; i < n; i++) {
    b.img.push_back(build_plan(p, in + (size_t)i * n_in, n_in, out + (size_t)i * n_out, n_out, true));
    const RunPlan &r = b.img.back();
    const RunPlan &r0 = b.img[0];
    if (i == 0) {
      for (const Launch &L : r.launches)
        if (!L.fused || L.key.otptb)
          fail(WT_EUNSUPPORTED, "batched runs need a warp-tiled schedule whose groups all fuse");
    } else {
      bool same = r.launches.size() == r0.launches.size();
      for (size_t l = 0; same && l < r.launches.size(); l++) same = r.launches[l].kname == r0.launches[l].kname;
      if (!same) fail(WT_EINVAL, "images of a batch must share channels and dtypes");
    }
    const int64_t off = align256(b.ws_bytes);
    b.ws_off.push_back(off);
    b.ws_bytes = off + r.ws_bytes;
  }
  const RunPlan &r0 = b.img[0];
  b.launches.resize(r0.launches.size());
  b.tiles.resize(r0.launches.size());
  for (size_t l = 0; l < r0.launches.size(); l++) {
    Launch L = r0.launches[l];
    L.key.persistent = true;
    L.kname = kernel_name(p, L.key, true, L.geom.n_gather > 0);
    std::vector<int32_t> &t = b.tiles[l];
    int64_t total = 0;
    for (int i = 0; i < n; i++) total += b.img[i].launches[l].n_tiles;
    if (total > (1ll << 30)) fail(WT_EUNSUPPORTED, "too many tiles in a batch");
    t.reserve((size_t)total * 4);
    // image by image, each plane row-major: neighbouring tiles share halo
    // rows in L2
    for (int i = 0; i < n; i++) {
      const Launch &Li = b.img[i].launches[l];
      for (int ch = 0; ch < Li.geom.channels; ch++)
        for (int ty = 0; ty < Li.tiles_y; ty++)
          for (int tx = 0; tx < Li.tiles_x; tx++) t.insert(t.end(), {i, tx, ty, ch});
    }
    L.n_tiles = (int)total;
    L.grid[0] = (unsigned)((total + L.key.nw - 1) / L.key.nw);
    b.launches[l] = L;
  }
  return b;
}

// Argument block of image i for batched launch l (ws: the image's slice of
// the workspace, or null for introspection).
KernelArgs batch_image_args(const Pipeline &p, const BatchPlan &b, int l, int i, char *ws, bool encode_tmaps) {
  KernelArgs a;
  fill_args(p, b.img[i], b.img[i].launches[l], ws, a, encode_tmaps);
  return a;
}

void run_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n, cudaStream_t stream) {
  int dev = 0;
  check_rt(cudaGetDevice(&dev), "cudaGetDevice");
  const int n_in = (int)p.in_channels.size(), n_out = (int)p.outputs.size();
  std::string key((const char *)in, sizeof(wt_image) * (size_t)n * n_in);
  key.append((const char *)out, sizeof(wt_image) * (size_t)n * n_out);
  const Driver &drv = driver();
  if (p.batch && p.ws && p.batch->device == dev && p.batch->sched_version == p.sched_version &&
      p.batch->ws_generation == p.ws->generation && p.batch->key == key) {
    CachedRun &c = p.batch->run;
    for (size_t i = 0; i < c.functions.size(); i++) {
      void *params[] = {&c.args[i]};
      check_cu(drv.launchKernel((CUfunction)c.functions[i], c.grid[3 * i], c.grid[3 * i + 1], c.grid[3 * i + 2],
                                (unsigned)c.block[i], 1, 1, (unsigned)c.smem[i], (CUstream)stream, params, nullptr),
               "cuLaunchKernel");
    }
    return;
  }
  BatchPlan b = build_batch(p, in, out, n);
  if ((int)b.launches.size() > kMaxLaunches) fail(WT_EUNSUPPORTED, "too many launches per batch");
  Workspace &w = workspace(p, b.ws_bytes);
  // device tables: per launch, n argument blocks then the tile list
  std::vector<int64_t> tab_off(b.launches.size()), tile_off(b.launches.size());
  int64_t bytes = 0;
  for (size_t l = 0; l < b.launches.size(); l++) {
    tab_off[l] = align256(bytes);
    bytes = tab_off[l] + (int64_t)n * (int64_t)sizeof(KernelArgs);
    tile_off[l] = align256(bytes);
    bytes = tile_off[l] + (int64_t)b.tiles[l].size() * 4;
  }
  auto bc = std::make_shared<BatchCache>();
  bc->device = dev;
  if (dev_alloc(&bc->table, (size_t)bytes) != cudaSuccess) {
    cudaGetLastError();
    fail(WT_ENOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of batch tables");
  }
  bc->table_bytes = bytes;
  std::vector<char> host((size_t)bytes, 0);
  for (size_t l = 0; l < b.launches.size(); l++) {
    for (int i = 0; i < n; i++) {
      KernelArgs a = batch_image_args(p, b, (int)l, i, w.base ? w.base + b.ws_off[i] : nullptr, true);
      memcpy(host.data() + tab_off[l] + (int64_t)i * sizeof(KernelArgs), &a, sizeof a);
    }
    memcpy(host.data() + tile_off[l], b.tiles[l].data(), b.tiles[l].size() * 4);
  }
  // the tables must be on the device before the first launch reads them;
  // synchronous: this is the once-per-batch-shape set-up
  check_rt(cudaMemcpyAsync(bc->table, host.data(), (size_t)bytes, cudaMemcpyHostToDevice, stream),
           "cudaMemcpyAsync(batch tables)");
  check_rt(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
  CachedRun &c = bc->run;
  int sms = 0;
  check_rt(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  for (size_t l = 0; l < b.launches.size(); l++) {
    Launch &L = b.launches[l];
    Kernel &k = get_kernel(p, L, dev);
    if (L.smem > 48 * 1024)
      check_cu(drv.funcSetAttribute((CUfunction)k.function, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, L.smem),
               "cuFuncSetAttribute");
    int per_sm = 0;
    check_cu(drv.occupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (CUfunction)k.function, L.block, (size_t)L.smem),
             "cuOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) fail(WT_EUNSUPPORTED, "group kernel cannot be resident (registers/shared memory)");
    L.grid[0] = std::min<unsigned>(L.grid[0], (unsigned)(per_sm * sms));
    KernelArgs a;
    memset(&a, 0, sizeof a);
    a.n_tiles = L.n_tiles;
    a.n_images = n;
    a.tile_table = (const int32_t *)((char *)bc->table + tile_off[l]);
    a.img_tab = (char *)bc->table + tab_off[l];
    a.err = w.err;
    a.queue = queue_counters(w.err, (int)l);
    c.functions.push_back(k.function);
    c.args.push_back(a);
    c.grid.insert(c.grid.end(), {L.grid[0], 1u, 1u});
    c.block.push_back(L.block);
    c.smem.push_back(L.smem);
  }
  for (size_t i = 0; i < c.functions.size(); i++) {
    void *params[] = {&c.args[i]};
    check_cu(drv.launchKernel((CUfunction)c.functions[i], c.grid[3 * i], 1, 1, (unsigned)c.block[i], 1, 1,
                              (unsigned)c.smem[i], (CUstream)stream, params, nullptr),
             "cuLaunchKernel");
  }
  bc->sched_version = p.sched_version;
  bc->ws_generation = w.generation;
  bc->key = std::move(key);
  if (p.batch) check_rt(cudaStreamSynchronize(stream), "cudaStreamSynchronize");  // old tables may be in use
  p.batch = bc;
}

}  // namespace wt
