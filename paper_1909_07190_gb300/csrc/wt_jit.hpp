// Driver-API entry points and run-time compilation (jit.cpp).
#pragma once

#include <cuda.h>

#include <string>

namespace wt {

struct Driver {
  bool ok = false;
  CUresult (*moduleLoadData)(CUmodule *, const void *) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction *, CUmodule, const char *) = nullptr;
  CUresult (*moduleUnload)(CUmodule) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           unsigned, CUstream, void **, void **) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*funcGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
  CUresult (*tensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill) = nullptr;
  CUresult (*getErrorString)(CUresult, const char **) = nullptr;
  CUresult (*occupancyMaxActiveBlocksPerMultiprocessor)(int *, CUfunction, int, size_t) = nullptr;
};

const Driver &driver();
void check_cu(int rc, const char *what);
void check_rt(int rc, const char *what);
// NVRTC -> CUBIN for sm_103a, with an on-disk cache keyed by source+options.
std::string compile_cubin(const std::string &src, const std::string &name, int max_regs);

}  // namespace wt
