// jit.hpp -- NVRTC compilation of generated kernels for sm_103a and their
// launch through the CUDA driver API.
#pragma once

#include <cuda.h>

#include <string>
#include <vector>
#include <unordered_map>

namespace dfs {

struct Driver {  // driver entry points, resolved through the runtime at first use
  CUresult (*ModuleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*ModuleUnload)(CUmodule) = nullptr;
  CUresult (*ModuleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*LaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           CUstream, void**, void**) = nullptr;
  CUresult (*LaunchCooperativeKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                                      unsigned, CUstream, void**) = nullptr;
  CUresult (*OccupancyMaxActiveBlocksPerMultiprocessor)(int*, CUfunction, int, size_t) = nullptr;
  CUresult (*FuncGetAttribute)(int*, CUfunction_attribute, CUfunction) = nullptr;
  CUresult (*FuncSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*GetErrorString)(CUresult, const char**) = nullptr;
  bool loaded = false;
};

// Loads the entry points; returns false with a message on failure.
bool driver_load(Driver& d, std::string& err);

struct Compiled {
  CUmodule module = nullptr;
  CUfunction fn = nullptr;
  int regs = 0;
  int occupancy = 0;  // resident CTAs per SM at the block size and dynamic shared memory
  int dyn_smem = 0;   // dynamic shared memory per CTA the kernel is launched with
  double compile_s = 0.0;
  bool from_disk = false;
};

class Jit {
 public:
  // `device_source` is the text of dfs_device.cuh.  `arch` e.g. "sm_103a".
  Jit(Driver* drv, std::string arch, std::string cache_dir);
  ~Jit();
  // Compiles (or fetches) the kernel `name` from `source`, to be launched with
  // `dyn_smem` bytes of dynamic shared memory per CTA; returns nullptr and
  // sets `err` on failure.
  const Compiled* get(const std::string& source, const std::string& name, int block, std::string& err,
                      int dyn_smem = 0);
  // NVRTC only (no device needed): returns the cubin size, 0 on failure.
  size_t compile_only(const std::string& source, const std::string& name, std::string& err);
  double compile_seconds() const { return compile_s_; }
  int compiles() const { return compiles_; }
  int hits() const { return hits_; }
  int disk_hits() const { return disk_hits_; }

 private:
  Driver* drv_;
  std::string arch_, cache_dir_;
  std::unordered_map<std::string, Compiled> cache_;
  bool nvrtc(const std::string& source, const std::string& name, std::vector<char>& cubin, std::string& err);
  double compile_s_ = 0.0;
  int compiles_ = 0, hits_ = 0, disk_hits_ = 0;
};

extern const char* const kDeviceSource;  // embedded dfs_device.cuh

}  // namespace dfs
