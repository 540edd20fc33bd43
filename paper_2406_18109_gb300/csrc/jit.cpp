// jit.cpp -- NVRTC compilation for sm_103a, an in-memory and optional on-disk
// cubin cache, and the CUDA driver entry points used to load and launch.
//
// Generated kernels are compiled once per distinct source (isomorphic windows
// produce identical source, Section 5.2), so steady-state iterations launch
// cached kernels.  A disk cache keeps cubins across processes, the production
// follow-up the paper suggests at the end of Section 7.2.
#include "jit.hpp"

#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <fstream>
#include <functional>
#include <sstream>
#include <vector>

namespace dfs {

#include "dfs_device_src.inc"  // defines kDeviceSourceText (generated at build time)

const char* const kDeviceSource = kDeviceSourceText;

template <typename F>
static bool resolve(const char* name, F& fp, std::string& err) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
    err = std::string("cannot resolve driver entry point ") + name + ": " + cudaGetErrorString(e);
    return false;
  }
  fp = reinterpret_cast<F>(p);
  return true;
}

bool driver_load(Driver& d, std::string& err) {
  if (d.loaded) return true;
  bool ok = resolve("cuModuleLoadData", d.ModuleLoadData, err) &&
            resolve("cuModuleUnload", d.ModuleUnload, err) &&
            resolve("cuModuleGetFunction", d.ModuleGetFunction, err) &&
            resolve("cuLaunchKernel", d.LaunchKernel, err) &&
            resolve("cuLaunchCooperativeKernel", d.LaunchCooperativeKernel, err) &&
            resolve("cuOccupancyMaxActiveBlocksPerMultiprocessor", d.OccupancyMaxActiveBlocksPerMultiprocessor,
                    err) &&
            resolve("cuFuncGetAttribute", d.FuncGetAttribute, err) &&
            resolve("cuFuncSetAttribute", d.FuncSetAttribute, err) &&
            resolve("cuGetErrorString", d.GetErrorString, err);
  d.loaded = ok;
  return ok;
}

Jit::Jit(Driver* drv, std::string arch, std::string cache_dir)
    : drv_(drv), arch_(std::move(arch)), cache_dir_(std::move(cache_dir)) {}

Jit::~Jit() {
  for (auto& kv : cache_)
    if (kv.second.module && drv_->ModuleUnload) drv_->ModuleUnload(kv.second.module);
}

static std::string hex(size_t h) {
  char b[32];
  snprintf(b, sizeof b, "%016zx", h);
  return b;
}

static const char* const kOpts[] = {"-std=c++17", "-default-device", "-lineinfo", "--extra-device-vectorization"};

bool Jit::nvrtc(const std::string& source, const std::string& name, std::vector<char>& cubin, std::string& err) {
  const std::string opt_arch = "--gpu-architecture=" + arch_;
  std::vector<const char*> opts = {opt_arch.c_str()};
  for (const char* o : kOpts) opts.push_back(o);
  nvrtcProgram prog;
  const char* hdr_src[] = {kDeviceSource};
  const char* hdr_name[] = {"dfs_device.cuh"};
  nvrtcResult r = nvrtcCreateProgram(&prog, source.c_str(), (name + ".cu").c_str(), 1, hdr_src, hdr_name);
  if (r != NVRTC_SUCCESS) {
    err = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
    return false;
  }
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  if (r != NVRTC_SUCCESS) {
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    err = std::string("NVRTC failed to compile ") + name + ": " + nvrtcGetErrorString(r) + "\n" + log;
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t cs = 0;
  nvrtcGetCUBINSize(prog, &cs);
  cubin.resize(cs);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return true;
}

size_t Jit::compile_only(const std::string& source, const std::string& name, std::string& err) {
  std::vector<char> cubin;
  const auto t0 = std::chrono::steady_clock::now();
  if (!nvrtc(source, name, cubin, err)) return 0;
  compile_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  ++compiles_;
  return cubin.size();
}

const Compiled* Jit::get(const std::string& source, const std::string& name, int block, std::string& err,
                         int dyn_smem) {
  auto it = cache_.find(source);
  if (it != cache_.end()) {
    ++hits_;
    return &it->second;
  }
  const auto t0 = std::chrono::steady_clock::now();
  int major = 0, minor = 0;
  nvrtcVersion(&major, &minor);
  std::string fingerprint = source + "|" + arch_ + "|" + std::to_string(major) + "." + std::to_string(minor) +
                            "|" + kDeviceSource;
  for (const char* o : kOpts) fingerprint += std::string("|") + o;
  const std::string disk_path =
      cache_dir_.empty() ? std::string() : cache_dir_ + "/" + name + "_" + hex(std::hash<std::string>{}(fingerprint)) + ".cubin";

  std::vector<char> cubin;
  bool from_disk = false;
  if (!disk_path.empty()) {
    std::ifstream f(disk_path, std::ios::binary);
    if (f) {
      cubin.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
      from_disk = !cubin.empty();
    }
  }
  if (!from_disk) {
    if (!nvrtc(source, name, cubin, err)) return nullptr;
    if (!disk_path.empty()) {
      const std::string tmp = disk_path + ".tmp" + hex((size_t)this);
      std::ofstream f(tmp, std::ios::binary);
      if (f) {
        f.write(cubin.data(), (std::streamsize)cubin.size());
        f.close();
        std::rename(tmp.c_str(), disk_path.c_str());
      }
    }
  }
  Compiled c;
  c.from_disk = from_disk;
  CUresult cr = drv_->ModuleLoadData(&c.module, cubin.data());
  if (cr == CUDA_SUCCESS) cr = drv_->ModuleGetFunction(&c.fn, c.module, name.c_str());
  if (cr != CUDA_SUCCESS) {
    const char* s = nullptr;
    drv_->GetErrorString(cr, &s);
    err = std::string("loading ") + name + ": " + (s ? s : "unknown driver error");
    return nullptr;
  }
  drv_->FuncGetAttribute(&c.regs, CU_FUNC_ATTRIBUTE_NUM_REGS, c.fn);
  if (dyn_smem > 0) {
    cr = drv_->FuncSetAttribute(c.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, dyn_smem);
    if (cr != CUDA_SUCCESS) {
      const char* s = nullptr;
      drv_->GetErrorString(cr, &s);
      err = std::string("dynamic shared memory of ") + name + ": " + (s ? s : "unknown driver error");
      drv_->ModuleUnload(c.module);
      return nullptr;
    }
  }
  c.dyn_smem = dyn_smem;
  drv_->OccupancyMaxActiveBlocksPerMultiprocessor(&c.occupancy, c.fn, block, (size_t)dyn_smem);
  const auto t1 = std::chrono::steady_clock::now();
  c.compile_s = std::chrono::duration<double>(t1 - t0).count();
  compile_s_ += c.compile_s;
  if (from_disk)
    ++disk_hits_;
  else
    ++compiles_;
  auto ins = cache_.emplace(source, c);
  return &ins.first->second;
}

}  // namespace dfs
