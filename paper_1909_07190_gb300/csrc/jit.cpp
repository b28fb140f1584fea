// Run-time compilation of generated group kernels with NVRTC (sm_103a CUBIN)
// and module loading through the CUDA driver API.  Driver entry points are
// resolved through the runtime (cudaGetDriverEntryPointByVersion), so the
// library loads on machines without a GPU driver; they are needed only
// when a kernel is compiled or launched.
#include <dlfcn.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>

#include "wt_internal.hpp"
#include "wt_jit.hpp"

namespace wt {

static Driver g_drv;
static std::once_flag g_drv_once;
static std::string g_drv_err;

#define WT_RESOLVE(name, field)                                                                 \
  do {                                                                                           \
    cudaDriverEntryPointQueryResult q;                                                           \
    void *fp = nullptr;                                                                          \
    if (cudaGetDriverEntryPointByVersion(#name, &fp, 12080, cudaEnableDefault, &q) !=           \
            cudaSuccess ||                                                                       \
        q != cudaDriverEntryPointSuccess || !fp) {                                               \
      g_drv_err = "cannot resolve driver entry point " #name;                                    \
      return;                                                                                    \
    }                                                                                            \
    g_drv.field = reinterpret_cast<decltype(g_drv.field)>(fp);                                   \
  } while (0)

const Driver &driver() {
  std::call_once(g_drv_once, [] {
    WT_RESOLVE(cuModuleLoadData, moduleLoadData);
    WT_RESOLVE(cuModuleGetFunction, moduleGetFunction);
    WT_RESOLVE(cuModuleUnload, moduleUnload);
    WT_RESOLVE(cuLaunchKernel, launchKernel);
    WT_RESOLVE(cuFuncSetAttribute, funcSetAttribute);
    WT_RESOLVE(cuFuncGetAttribute, funcGetAttribute);
    WT_RESOLVE(cuTensorMapEncodeTiled, tensorMapEncodeTiled);
    WT_RESOLVE(cuGetErrorString, getErrorString);
    WT_RESOLVE(cuOccupancyMaxActiveBlocksPerMultiprocessor, occupancyMaxActiveBlocksPerMultiprocessor);
    g_drv.ok = true;
  });
  if (!g_drv.ok) fail(WT_ECUDA, g_drv_err.empty() ? "CUDA driver unavailable" : g_drv_err);
  return g_drv;
}

void check_cu(int rc, const char *what) {
  if (rc == CUDA_SUCCESS) return;
  const char *s = nullptr;
  if (g_drv.getErrorString) g_drv.getErrorString((CUresult)rc, &s);
  fail(WT_ECUDA, std::string(what) + ": " + (s ? s : "driver error ") + "(" + std::to_string(rc) + ")");
}

void check_rt(int rc, const char *what) {
  if (rc == cudaSuccess) return;
  fail(WT_ECUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)rc));
}

// compiled kernels of this process (NVRTC runs once per kernel text)
static std::mutex g_cubin_mu;
static std::map<std::string, std::string> g_cubins;

// On-disk cubin cache: $WT_CACHE_DIR, else _build/kernel_cache beside the
// library itself (the package directory), so that a build keeps its files
// in its own tree.
static std::string cache_dir() {
  const char *e = getenv("WT_CACHE_DIR");
  if (e && *e) return e;
  Dl_info info;
  if (dladdr((const void *)&cache_dir, &info) && info.dli_fname) {
    std::string lib(info.dli_fname);
    const size_t slash = lib.rfind('/');
    if (slash != std::string::npos) return lib.substr(0, slash) + "/_build/kernel_cache";
  }
  return "_build/kernel_cache";
}

static void mkdirs(const std::string &d) {
  std::string cur;
  for (size_t i = 0; i < d.size(); i++) {
    cur += d[i];
    if (d[i] == '/' || i + 1 == d.size()) mkdir(cur.c_str(), 0755);
  }
}

std::string compile_cubin(const std::string &src, const std::string &name, int max_regs) {
  int major = 0, minor = 0;
  nvrtcVersion(&major, &minor);
  std::vector<std::string> opts = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG"};
  if (max_regs > 0) opts.push_back("-maxrregcount=" + std::to_string(max_regs));
  uint64_t h = fnv1a(src.data(), src.size());
  for (auto &o : opts) h = fnv1a(o.data(), o.size(), h);
  h = fnv1a(&major, sizeof major, h);
  h = fnv1a(&minor, sizeof minor, h);
  char hex[32];
  snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
  std::string dir = cache_dir();
  std::string path = dir + "/" + name + "_" + hex + ".cubin";
  {
    std::lock_guard<std::mutex> lk(g_cubin_mu);
    auto it = g_cubins.find(name + "_" + hex);
    if (it != g_cubins.end()) return it->second;
  }
  auto remember = [&](const std::string &b) {
    std::lock_guard<std::mutex> lk(g_cubin_mu);
    if (g_cubins.size() > 512) g_cubins.clear();
    g_cubins[name + "_" + hex] = b;
  };
  if (!getenv("WT_NO_DISK_CACHE")) {
    std::ifstream f(path, std::ios::binary);
    if (f) {
      std::stringstream ss;
      ss << f.rdbuf();
      std::string b = ss.str();
      if (!b.empty()) {
        remember(b);
        return b;
      }
    }
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), (name + ".cu").c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS)
    fail(WT_ECOMPILE, "nvrtcCreateProgram failed");
  std::vector<const char *> cop;
  for (auto &o : opts) cop.push_back(o.c_str());
  nvrtcResult rc = nvrtcCompileProgram(prog, (int)cop.size(), cop.data());
  size_t logn = 0;
  nvrtcGetProgramLogSize(prog, &logn);
  std::string log(logn, '\0');
  if (logn) nvrtcGetProgramLog(prog, &log[0]);
  if (rc != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    if (log.size() > 4000) log = log.substr(0, 4000);
    fail(WT_ECOMPILE, "NVRTC failed for " + name + ": " + log);
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::string cubin(n, '\0');
  nvrtcGetCUBIN(prog, &cubin[0]);
  nvrtcDestroyProgram(&prog);
  if (!getenv("WT_NO_DISK_CACHE")) {
    mkdirs(dir);
    std::string tmp = path + "." + std::to_string(getpid()) + "." +
                      std::to_string(std::hash<std::thread::id>()(std::this_thread::get_id())) + ".tmp";
    std::ofstream f(tmp, std::ios::binary);
    if (f) {
      f.write(cubin.data(), (std::streamsize)cubin.size());
      f.close();
      rename(tmp.c_str(), path.c_str());
    }
  }
  remember(cubin);
  return cubin;
}

}  // namespace wt
