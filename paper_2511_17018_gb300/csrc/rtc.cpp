// Run-time compilation of the fit (Sec. 5).
//
// The fit kernel is compiled with NVRTC for the handle's time-frame constants:
// the field (kappa), the cluster variance, the initial factor, the sin(phi)
// limit and the number of pad rows become compile-time constants, and the
// row and rotation tables become initialised constant memory, so the compiler
// folds them into the code.  The source is the same device code the library
// compiles ahead of time (fit_core.cuh, embedded into the library by the build),
// compiled with the same flags for the mode, so a kernel compiled at run time
// computes what the ahead-of-time one computes for the same constants.
//
// Each distinct source (constants, mode, launch shape, record / batched-frame
// variant) is compiled once per process and kept; with a cache directory the
// CUBIN is also written to and read from disk, so later processes skip the
// compilation.  NVRTC is loaded on first use (dlopen); without it, run-time
// compilation reports TPCFIT_ERTC and the ahead-of-time kernels stay usable.
#include <dlfcn.h>
#include <nvrtc.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace tpcfit {

// Embedded device sources (generated by the build from csrc/).
extern const int kRtcSourceCount;
extern const char* const kRtcSourceNames[];
extern const char* const kRtcSources[];

namespace {

struct NvrtcApi {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok = false;
};

const NvrtcApi& nvrtc() {
  static NvrtcApi api;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {getenv("TPCFIT_NVRTC"), "libnvrtc.so.13", "libnvrtc.so",
                           "/usr/local/cuda/lib64/libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* n : names) {
      if (n && *n && (h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    }
    if (!h) return;
    api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
    api.add_name = reinterpret_cast<decltype(api.add_name)>(dlsym(h, "nvrtcAddNameExpression"));
    api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
    api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
    api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    api.lowered = reinterpret_cast<decltype(api.lowered)>(dlsym(h, "nvrtcGetLoweredName"));
    api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    api.ok = api.create && api.add_name && api.compile && api.log_size && api.log && api.cubin_size && api.cubin &&
             api.lowered && api.destroy;
  });
  return api;
}

// Exact text of a float (C99 hexadecimal floating point).
std::string hexf(float v) {
  char b[64];
  snprintf(b, sizeof b, "%af", (double)v);
  return b;
}

template <typename T, typename F>
void append_list(std::string& s, const T* v, int n, F fmt) {
  s += "{";
  for (int i = 0; i < n; ++i) {
    if (i) s += ", ";
    s += fmt(v[i]);
  }
  s += "}";
}

uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

struct Compiled {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  std::unordered_map<int, int> grid;  // per device: resident blocks over all SMs
};

std::mutex g_mu;
std::unordered_map<std::string, Compiled*> g_cache;
std::string g_log;
std::atomic<long long> g_compiles{0};

std::vector<std::string> options(bool det) {
  std::vector<std::string> o = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
  if (det) {
    o.insert(o.end(), {"-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"});
  } else {
    o.insert(o.end(), {"-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"});
  }
  return o;
}

bool read_file(const std::string& path, std::vector<char>& out) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  fseek(f, 0, SEEK_END);
  const long n = ftell(f);
  fseek(f, 0, SEEK_SET);
  out.resize(n > 0 ? (size_t)n : 0);
  const bool ok = n > 0 && fread(out.data(), 1, (size_t)n, f) == (size_t)n;
  fclose(f);
  return ok;
}

// Write via a temporary name and rename, so that concurrent processes never
// read a partial file.
void write_file(const std::string& path, const std::vector<char>& data) {
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
  fclose(f);
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

// NVRTC: source -> CUBIN and the lowered name of `expr`.
tpcfit_status compile(const std::string& src, const std::string& expr, bool det, std::vector<char>& cubin,
                      std::string& lowered) {
  const NvrtcApi& api = nvrtc();
  if (!api.ok) {
    g_log = "NVRTC library not found";
    return TPCFIT_ERTC;
  }
  nvrtcProgram prog = nullptr;
  if (api.create(&prog, src.c_str(), "tpcfit_rtc.cu", kRtcSourceCount, kRtcSources, kRtcSourceNames) !=
      NVRTC_SUCCESS) {
    g_log = "nvrtcCreateProgram failed";
    return TPCFIT_ERTC;
  }
  api.add_name(prog, expr.c_str());
  const std::vector<std::string> o = options(det);
  std::vector<const char*> argv;
  for (const std::string& x : o) argv.push_back(x.c_str());
  const nvrtcResult r = api.compile(prog, (int)argv.size(), argv.data());
  size_t ls = 0;
  api.log_size(prog, &ls);
  std::string log(ls, '\0');
  if (ls) api.log(prog, &log[0]);
  g_log = log;
  tpcfit_status st = TPCFIT_OK;
  if (r != NVRTC_SUCCESS) {
    st = TPCFIT_ERTC;
  } else {
    size_t n = 0;
    const char* name = nullptr;
    if (api.cubin_size(prog, &n) != NVRTC_SUCCESS || n == 0 || api.lowered(prog, expr.c_str(), &name) != NVRTC_SUCCESS ||
        !name) {
      st = TPCFIT_ERTC;
    } else {
      cubin.resize(n);
      if (api.cubin(prog, cubin.data()) != NVRTC_SUCCESS) st = TPCFIT_ERTC;
      lowered = name;
    }
  }
  api.destroy(&prog);
  g_compiles.fetch_add(1);
  return st;
}

}  // namespace

bool rtc_available() { return nvrtc().ok; }
long long rtc_compile_count() { return g_compiles.load(); }
const char* rtc_log() { return g_log.c_str(); }

std::string rtc_fit_source(const GeoConst& g, bool det) {
  std::string s;
  s += "// fit kernel specialised for one time frame (generated)\n";
  s += "#define TPCFIT_RTC 1\n";
  s += det ? "#define TPCFIT_DET 1\n" : "#define TPCFIT_DET 0\n";
  s += "#define TPCFIT_NS rtc\n";
  s += "#include \"kernel_abi.h\"\n";
  s += "namespace tpcfit {\nnamespace rtc {\n";
  s += "struct GeoFold {\n";
  s += "  float row_x[kMaxRows];\n  float rot_c[kNSide * kNSide];\n  float rot_s[kNSide * kNSide];\n";
  s += "  static constexpr float kappa = " + hexf(g.kappa) + ";\n";
  s += "  static constexpr float v_meas = " + hexf(g.v_meas) + ";\n";
  s += "  static constexpr float sqrt_v = " + hexf(g.sqrt_v) + ";\n";
  s += "  static constexpr float l0 = " + hexf(g.l0) + ";\n";
  s += "  static constexpr float max_snp = " + hexf(g.max_snp) + ";\n";
  s += "  static constexpr int32_t n_rows = " + std::to_string(g.n_rows) + ";\n";
  s += "  static constexpr int32_t mat = " + std::to_string(g.mat) + ";\n";
  s += "  static constexpr float x0_inv = " + hexf(g.x0_inv) + ";\n";
  s += "  static constexpr float dedx = " + hexf(g.dedx) + ";\n";
  s += "  static constexpr float mass2 = " + hexf(g.mass2) + ";\n";
  s += "  static constexpr float d_row = " + hexf(g.d_row) + ";\n";
  s += "  static constexpr int32_t field = " + std::to_string(g.field) + ";\n";
  s += "  static constexpr float f_r = " + hexf(g.f_r) + ";\n";
  s += "  static constexpr float f_z = " + hexf(g.f_z) + ";\n";
  s += "};\n";
  s += "__constant__ GeoFold c_geo = {";
  append_list(s, g.row_x, kMaxRows, hexf);
  s += ", ";
  append_list(s, g.rot_c, kNSide * kNSide, hexf);
  s += ", ";
  append_list(s, g.rot_s, kNSide * kNSide, hexf);
  s += "};\n}  // namespace rtc\n}  // namespace tpcfit\n";
  s += "#include \"fit_core.cuh\"\n";
  return s;
}

namespace {

// Key, source and kernel name of the fit variant.
struct Variant {
  std::string src, expr, key;
};

Variant variant(const GeoConst& g, bool det, int rps, int warps, bool record, bool frames, int form) {
  Variant v;
  v.src = rtc_fit_source(g, det);
  v.expr = "tpcfit::rtc::fit_kernel<" + std::to_string(rps) + ", " + std::to_string(warps) + ", " +
           std::to_string(fit_min_blocks(rps, warps)) + ", " + (record ? "true" : "false") + ", " +
           (frames ? "true" : "false") + ", " + std::to_string((g.mat ? 1 : 0) | (g.field ? 2 : 0)) + ", " +
           std::to_string(form) + ">";
  std::string opt;
  for (const std::string& x : options(det)) opt += x + " ";
  char keyb[32];
  snprintf(keyb, sizeof keyb, "%016llx", (unsigned long long)fnv1a(v.expr, fnv1a(opt, fnv1a(v.src))));
  v.key = keyb;
  return v;
}

// CUBIN of a variant: from the cache directory if it holds one, else compiled
// (and then stored there).
tpcfit_status cubin_of(const Variant& v, bool det, const char* cache_dir, std::vector<char>& cubin,
                       std::string& lowered) {
  const std::string dir = cache_dir ? cache_dir : "";
  const std::string base = dir.empty() ? "" : dir + "/tpcfit_fit_" + v.key;
  if (!base.empty()) {
    std::vector<char> name;
    if (read_file(base + ".cubin", cubin) && read_file(base + ".name", name)) {
      lowered.assign(name.begin(), name.end());
      if (!lowered.empty()) return TPCFIT_OK;
    }
  }
  const tpcfit_status st = compile(v.src, v.expr, det, cubin, lowered);
  if (st != TPCFIT_OK) return st;
  if (!base.empty()) {
    write_file(base + ".cubin", cubin);
    write_file(base + ".name", std::vector<char>(lowered.begin(), lowered.end()));
  }
  return TPCFIT_OK;
}

}  // namespace

tpcfit_status rtc_build(const GeoConst& g, bool det, int rps, int warps, bool record, bool frames,
                        const char* cache_dir) {
  // the library's default factor: U-D in fast mode without material layers
  const Variant v = variant(g, det, rps, warps, record, frames, (!det && !g.mat) ? 1 : 0);
  std::vector<char> cubin;
  std::string lowered;
  return cubin_of(v, det, cache_dir, cubin, lowered);
}

tpcfit_status rtc_launch_fit(const GeoConst& g, bool det, int rps, int warps, const FitArgs& a, const char* cache_dir,
                             cudaStream_t s) {
  if (a.n_tracks <= 0) return TPCFIT_OK;
  const Variant v = variant(g, det, rps, warps, a.ck != nullptr, a.frame_base != nullptr,
                            (!det && !g.mat && a.form == 1) ? 1 : 0);
  const std::string& key = v.key;
  Compiled* c = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) c = it->second;
  }
  if (!c) {
    std::vector<char> cubin;
    std::string lowered;
    const tpcfit_status st = cubin_of(v, det, cache_dir, cubin, lowered);
    if (st != TPCFIT_OK) return st;
    Compiled* fresh = new Compiled();
    cudaError_t e = cudaLibraryLoadData(&fresh->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&fresh->kernel, fresh->lib, lowered.c_str());
    if (e != cudaSuccess) {
      if (fresh->lib) cudaLibraryUnload(fresh->lib);
      delete fresh;
      return TPCFIT_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
      g_cache[key] = fresh;
      c = fresh;
    } else {  // another thread got there first
      cudaLibraryUnload(fresh->lib);
      delete fresh;
      c = it->second;
    }
  }

  const int threads = warps * kWarp;
  const size_t smem = (size_t)kFitBlockSmemBytes + (size_t)warps * fit_warp_stage_bytes(rps);
  const void* fn = reinterpret_cast<const void*>(c->kernel);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  int grid = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = c->grid.find(dev);
    if (it != c->grid.end()) grid = it->second;
  }
  if (grid == 0) {
    int sms = 0, per_sm = 0;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (e != cudaSuccess || per_sm < 1) return TPCFIT_ECUDA;
    grid = sms * per_sm;
    std::lock_guard<std::mutex> lk(g_mu);
    c->grid[dev] = grid;
  }
  const int64_t chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t need = (chunks + warps - 1) / warps;
  const int blocks = (int)(need < grid ? need : grid);
  e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  FitArgs args = a;
  void* params[] = {&args};
  e = cudaLaunchKernel(fn, dim3(blocks), dim3(threads), params, smem, s);
  return e == cudaSuccess ? TPCFIT_OK : TPCFIT_ECUDA;
}

}  // namespace tpcfit
