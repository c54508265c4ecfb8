// pcpd_capi.cu -- the C ABI of libpcpd.so (declared in include/pcpd.h): handles, thresholds,
// time bookkeeping, tile plans and kernel launches for the bit-sliced PCPD sweep.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <nvtx3/nvToolsExt.h>

#include <type_traits>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/pcpd.h"
#include "pcpd_engine.cuh"
#include "pcpd_paper.cuh"

namespace {

// NVTX range around each public call that does device work (visible in profilers' timelines;
// free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

thread_local std::string g_err;

// Kernels this library has launched in this process (all threads).
std::atomic<unsigned long long> g_launches{0};

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? PCPD_ENOMEM : PCPD_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

constexpr uint64_t kTwo32 = 4294967296ull;

// Device allocation of the library's large buffers.  A request larger than the device's free
// memory is refused up front (PCPD_ENOMEM) rather than handed to cudaMalloc.  Tests can make
// the n-th such allocation of the process fail by setting PCPD_INJECT_ALLOC_FAILURE=n (host-
// side fault injection: nothing is allocated and the device is not touched).
std::atomic<long long> g_alloc_countdown{-2};   // -2: not read yet, -1: no injection

int dev_alloc(void **p, size_t bytes, const char *what) {
  long long c = g_alloc_countdown.load();
  if (c == -2) {
    const char *env = getenv("PCPD_INJECT_ALLOC_FAILURE");
    long long v = env ? atoll(env) : -1;
    g_alloc_countdown.compare_exchange_strong(c, v > 0 ? v : -1);
  }
  if (g_alloc_countdown.load() > 0 && --g_alloc_countdown == 0)
    return fail(PCPD_ENOMEM, "%s: injected allocation failure (%zu bytes)", what, bytes);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && bytes > free_b)
    return fail(PCPD_ENOMEM, "%s: %zu bytes requested, %zu free on the device", what, bytes, free_b);
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? PCPD_ENOMEM : PCPD_ECUDA, "%s: cudaMalloc(%zu): %s", what, bytes,
                cudaGetErrorString(e));
  return PCPD_OK;
}

// Rates of Eq. (1) as integer thresholds, evaluated in double exactly as written (the
// library is compiled with -ffp-contract=off, so no product is fused).
uint64_t floor_scaled(double x) {
  const double f = std::floor(x);
  if (f <= 0.0) return 0;
  if (f >= 4294967296.0) return kTwo32;
  return (uint64_t)f;
}

int thresholds(double p, double d, uint64_t *td, uint64_t *tda) {
  if (!(p >= 0.0 && p <= 1.0 && d >= 0.0 && d <= 1.0))
    return fail(PCPD_EINVAL, "p and d must lie in [0, 1] (p=%g, d=%g)", p, d);
  const uint64_t t_d = floor_scaled(d * 4294967296.0);
  double a = p * (1.0 - d);
  a = a * 4294967296.0;
  uint64_t t_da = t_d + floor_scaled(a);
  if (t_da > kTwo32) t_da = kTwo32;
  *td = t_d;
  *tda = t_da;
  return PCPD_OK;
}

// ceil(t*L/K), K = floor(L/W) windows of W sites (3 for the PCPD, n+1 for n-tuples): the
// sub-step at which MCS time t is reached.
uint64_t substep_of_time(uint32_t L, uint64_t t, uint32_t W = 3u) {
  const unsigned __int128 K = L / W;
  const unsigned __int128 num = (unsigned __int128)t * L;
  return (uint64_t)((num + K - 1) / K);
}

// Largest MCS time reached after n sub-steps: floor(n*K/L).
uint64_t time_of_substep(uint32_t L, uint64_t n, uint32_t W = 3u) {
  return (uint64_t)(((unsigned __int128)n * (L / W)) / L);
}

pcpdk::Thresholds split_thresholds(uint64_t td, uint64_t tda) {
  pcpdk::Thresholds T;
  T.td_full = td >= kTwo32;
  T.tda_full = tda >= kTwo32;
  T.td = (uint32_t)(T.td_full ? 0u : td);
  T.tda = (uint32_t)(T.tda_full ? 0u : tda);
  // lowest plane that matters: the lowest set bit of T (none for T = 0 or 2^32)
  T.lo_d = (T.td_full || T.td == 0u) ? 32u : (uint32_t)__builtin_ctz(T.td);
  T.lo_da = (T.tda_full || T.tda == 0u) ? 32u : (uint32_t)__builtin_ctz(T.tda);
  for (int m = 0; m < 32; ++m) {
    T.tmD[m] = (!T.td_full && ((T.td >> m) & 1u)) ? 0xFFFFFFFFu : 0u;
    T.tmA[m] = (!T.tda_full && ((T.tda >> m) & 1u)) ? 0xFFFFFFFFu : 0u;
  }
  return T;
}

int device_check() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0)
    return fail(PCPD_ENODEV, "no CUDA device (%s)", e == cudaSuccess ? "count 0" : cudaGetErrorString(e));
  int dev = 0, major = 0, minor = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  CU(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  // sm_103a code runs on compute capability 10.3 only (the "a" features do not carry over)
  if (major != 10 || minor != 3)
    return fail(PCPD_ENODEV, "device %d has compute capability %d.%d; the library is compiled for sm_103a (10.3)",
                dev, major, minor);
  return PCPD_OK;
}

int smem_optin(int *bytes) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return PCPD_OK;
}

// Static shared memory of the tile kernel (phase buffer + reduction slots), with margin.
constexpr size_t kStaticSmem = sizeof(uint32_t) * pcpdk::kPhiChunk + 34 * sizeof(unsigned int) + 256;

}  // namespace

// ------------------------------------------------------------------------------------------
struct pcpd {
  uint32_t L = 0, K = 0, S = 0, G = 0, pitch = 0;
  uint32_t W = 3;             // window width: tuple size + 1
  uint32_t g_base = 0;        // global index of the first group (pcpd_params.group0)
  double p = 0, d = 0;
  uint64_t seed = 0, td = 0, tda = 0;
  pcpdk::Thresholds T{};
  uint32_t k0 = 0, k1 = 0;
  int init = 0;
  bool per_sample = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t *buf[2] = {nullptr, nullptr};
  int cur = 0;
  bool own_mem = false;
  uint64_t n_now = 0, t_now = 0;
  // records
  std::vector<uint64_t> rec_times;
  unsigned long long *d_rec_total = nullptr;
  unsigned long long *d_rec_pairs = nullptr;
  uint32_t *d_rec_sample = nullptr;
  size_t rec_cap = 0;
  uint32_t *d_rec_sub = nullptr;
  size_t rec_sub_cap = 0;
  // plan (see make_plan)
  bool ring = true;
  uint32_t gpi = 1, threads = 0, core = 0, halo = 0, tau = 0, n_seg = 1;
  size_t tile_words = 0, dyn_smem = 0;
  int grid = 0;
  // engine scratch: per-tile epoch flags, work counter, error word
  uint32_t *d_done = nullptr;   // [tiles], then counter, then error word
  uint32_t tiles = 0;
  CUfunction jit_fn = nullptr;  // sweep compiled for this instance's thresholds, or null
};

namespace {

// The engine's dynamic shared-memory limit is a per-function, process-wide attribute: raise it
// once to the device maximum for both variants, so that handles with different tile sizes
// (and threads using them concurrently) never undercut one another.
std::mutex g_smem_mu;
bool g_smem_raised = false;

using SweepKernel = void (*)(const pcpdk::BatchParams);

// The sweep engine for single-instance or batched launches whose instances all have window
// width W (3, 4, 5), or a batch that mixes them (W = 0: read per instance).
SweepKernel sweep_kernel(bool batch, uint32_t W) {
  switch (W) {
    case 3: return batch ? pcpdk::k_sweep_persistent<true, 3> : pcpdk::k_sweep_persistent<false, 3>;
    case 4: return batch ? pcpdk::k_sweep_persistent<true, 4> : pcpdk::k_sweep_persistent<false, 4>;
    case 5: return batch ? pcpdk::k_sweep_persistent<true, 5> : pcpdk::k_sweep_persistent<false, 5>;
    default: return batch ? pcpdk::k_sweep_persistent<true, 0> : pcpdk::k_sweep_persistent<false, 3>;
  }
}

int raise_smem_limit() {
  std::lock_guard<std::mutex> lock(g_smem_mu);
  if (g_smem_raised) return PCPD_OK;
  int optin = 0;
  int rc = smem_optin(&optin);
  if (rc) return rc;
  for (int b = 0; b < 2; ++b)
    for (uint32_t W : {0u, 3u, 4u, 5u}) {
      const SweepKernel k = sweep_kernel(b != 0, W);
      cudaFuncAttributes fa;
      CU(cudaFuncGetAttributes(&fa, k));
      CU(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    }
  g_smem_raised = true;
  return PCPD_OK;
}

// ---- sweep specialised for one (T_D, T_DA) pair, compiled at run time ----
#include "pcpd_jit_src.inc"

// The runtime compiler and the driver calls it needs, resolved at run time so that the
// library loads (and the generic kernels run) even where either is missing.
struct JitApi {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
  nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
  nvrtcResult (*log_size)(nvrtcProgram, size_t *);
  nvrtcResult (*log)(nvrtcProgram, char *);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
  nvrtcResult (*cubin)(nvrtcProgram, char *);
  nvrtcResult (*destroy)(nvrtcProgram *);
  nvrtcResult (*add_name)(nvrtcProgram, const char *);
  nvrtcResult (*lowered_name)(nvrtcProgram, const char *, const char **);
  CUresult (*load)(CUmodule *, const void *);
  CUresult (*get_global)(CUdeviceptr *, size_t *, CUmodule, const char *);
  CUresult (*get_fn)(CUfunction *, CUmodule, const char *);
  CUresult (*get_attr)(int *, CUfunction_attribute, CUfunction);
  CUresult (*set_attr)(CUfunction, CUfunction_attribute, int);
  CUresult (*occupancy)(int *, CUfunction, int, size_t);
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                     void **, void **);
};

std::mutex g_jit_mu;
JitApi g_jit_api;
bool g_jit_api_tried = false;
// One runtime-compiled module: the single-instance entry, the batched entry (descriptors from
// the module's own constant table) and that table's device address.
struct JitEntry {
  CUfunction fn = nullptr, fn_batch = nullptr;
  CUdeviceptr c_inst = 0;
  size_t c_inst_bytes = 0;
};
std::map<std::tuple<int, uint32_t, uint32_t, uint32_t>, JitEntry> g_jit;

template <typename F>
bool driver_fn(const char *name, F *out) {
  cudaDriverEntryPointQueryResult st;
  void *p = nullptr;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &st) != cudaSuccess ||
      st != cudaDriverEntryPointSuccess || !p)
    return false;
  *out = reinterpret_cast<F>(p);
  return true;
}

const JitApi &jit_api() {   // call with g_jit_mu held
  if (g_jit_api_tried) return g_jit_api;
  g_jit_api_tried = true;
  JitApi a;
  void *lib = dlopen("libnvrtc.so.13", RTLD_NOW | RTLD_LOCAL);
  if (!lib) lib = dlopen("libnvrtc.so", RTLD_NOW | RTLD_LOCAL);
  if (!lib) return g_jit_api;
  bool ok = true;
  auto sym = [&](const char *n, auto *f) {
    void *p = dlsym(lib, n);
    ok = ok && p;
    *f = reinterpret_cast<std::remove_pointer_t<decltype(f)>>(p);
  };
  sym("nvrtcCreateProgram", &a.create);
  sym("nvrtcCompileProgram", &a.compile);
  sym("nvrtcGetProgramLogSize", &a.log_size);
  sym("nvrtcGetProgramLog", &a.log);
  sym("nvrtcGetCUBINSize", &a.cubin_size);
  sym("nvrtcGetCUBIN", &a.cubin);
  sym("nvrtcDestroyProgram", &a.destroy);
  sym("nvrtcAddNameExpression", &a.add_name);
  sym("nvrtcGetLoweredName", &a.lowered_name);
  ok = ok && driver_fn("cuModuleLoadData", &a.load) && driver_fn("cuModuleGetFunction", &a.get_fn) &&
       driver_fn("cuModuleGetGlobal", &a.get_global) &&
       driver_fn("cuFuncGetAttribute", &a.get_attr) && driver_fn("cuFuncSetAttribute", &a.set_attr) &&
       driver_fn("cuOccupancyMaxActiveBlocksPerMultiprocessor", &a.occupancy) &&
       driver_fn("cuLaunchKernel", &a.launch);
  a.ok = ok;
  g_jit_api = a;
  return g_jit_api;
}

// Compile (once per device, threshold pair and window width) the engine with the thresholds
// and the window width as constants: the single-instance and the batched entry of one module.
int jit_entry(uint32_t td, uint32_t tda, uint32_t W, const JitEntry **out) {
#ifdef PCPD_DEBUG
  (void)td, (void)tda, (void)W, (void)out;
  return fail(PCPD_ECUDA, "debug builds run the generic sweep only (its checks live in this library)");
#endif
  int dev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaFree(nullptr));   // the runtime's primary context is current for the driver calls
  std::lock_guard<std::mutex> lock(g_jit_mu);
  const JitApi &J = jit_api();
  if (!J.ok) return fail(PCPD_ECUDA, "runtime compiler or driver entry points unavailable");
  auto key = std::make_tuple(dev, td, tda, W);
  auto it = g_jit.find(key);
  if (it != g_jit.end()) {
    *out = &it->second;
    return PCPD_OK;
  }
  nvrtcProgram prog;
  if (J.create(&prog, kJitSource, "pcpd_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return fail(PCPD_ECUDA, "nvrtcCreateProgram failed");
  static const char kTableExpr[] = "&pcpdk::c_inst";
  J.add_name(prog, kTableExpr);
  char dtd[64], dtda[64], dw[32];
  snprintf(dtd, sizeof dtd, "-DPCPD_JIT_TD=0x%08xu", td);
  snprintf(dtda, sizeof dtda, "-DPCPD_JIT_TDA=0x%08xu", tda);
  snprintf(dw, sizeof dw, "-DPCPD_JIT_W=%u", W);
  const char *opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", dtd, dtda, dw};
  const nvrtcResult rc = J.compile(prog, 6, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    J.log_size(prog, &n);
    std::string log(n, ' ');
    J.log(prog, &log[0]);
    J.destroy(&prog);
    return fail(PCPD_ECUDA, "runtime compile failed (%d): %.300s", (int)rc, log.c_str());
  }
  const char *lowered = nullptr;
  std::string table_name;
  if (J.lowered_name(prog, kTableExpr, &lowered) == NVRTC_SUCCESS && lowered) table_name = lowered;
  size_t cb = 0;
  J.cubin_size(prog, &cb);
  std::vector<char> cubin(cb);
  J.cubin(prog, cubin.data());
  J.destroy(&prog);
  CUmodule mod = nullptr;
  JitEntry e;
  if (J.load(&mod, cubin.data()) != CUDA_SUCCESS || J.get_fn(&e.fn, mod, "pcpd_jit_sweep") != CUDA_SUCCESS ||
      J.get_fn(&e.fn_batch, mod, "pcpd_jit_sweep_batch") != CUDA_SUCCESS)
    return fail(PCPD_ECUDA, "loading the runtime-compiled sweep failed");
  if (table_name.empty() || J.get_global(&e.c_inst, &e.c_inst_bytes, mod, table_name.c_str()) != CUDA_SUCCESS)
    e.fn_batch = nullptr;   // no descriptor table: batches keep the generic kernel
  int optin = 0, stat = 0;
  int rc2 = smem_optin(&optin);
  if (rc2) return rc2;
  for (CUfunction f : {e.fn, e.fn_batch}) {
    if (!f) continue;
    J.get_attr(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, f);
    if (J.set_attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, optin - stat) != CUDA_SUCCESS)
      return fail(PCPD_ECUDA, "setting the shared-memory limit of the runtime-compiled sweep failed");
  }
  auto ins = g_jit.emplace(key, e);   // modules stay loaded until the process exits
  *out = &ins.first->second;
  return PCPD_OK;
}

int jit_function(uint32_t td, uint32_t tda, uint32_t W, CUfunction *out) {
  const JitEntry *e = nullptr;
  const int rc = jit_entry(td, tda, W, &e);
  if (rc) return rc;
  *out = e->fn;
  return PCPD_OK;
}

// Tile plan.  Columns that fit in shared memory run as RING tiles (whole columns, gpi of them
// per CTA when they are short, so that a CTA has enough windows per sub-step); longer columns
// are cut into equal SEGMENT tiles with a halo of (W-1)*tau + W + 1 sites.  Modes:
//  kPlanPaired (a lone instance): SEGMENT tiles sized so that two CTAs of 256 threads share an
//    SM (one CTA's barriers and deferred-window tail overlap the other's first pass), tau =
//    64, and columns cut into enough tiles for every SM;
//  kPlanPairedBatch (batch and server members, which share one CTA shape per launch): every
//    tile, RING or SEGMENT, fits half an SM and CTAs have at most 256 threads, so a launch of
//    any mix of members runs two CTAs per SM;
//  kPlanOne (the allocation-free sweep, and the fallback of the others): one CTA of
//    kSweepThreads per SM holds the largest tile, tau = 128.
// No plan changes a result bit.
enum PlanMode { kPlanOne = 0, kPlanPaired = 1, kPlanPairedBatch = 2 };

int make_plan(pcpd_t *h, const pcpd_params *prm, PlanMode mode = kPlanOne) {
  const bool paired = mode != kPlanOne, batch = mode == kPlanPairedBatch;
  int optin = 0, dev = 0, sms = 0;
  int rc = smem_optin(&optin);
  if (rc) return rc;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t list_words = pcpdk::sweep_queue_words(32);
  const size_t avail_words = ((size_t)optin - kStaticSmem) / 4 - list_words;
  // shared memory each of two CTAs on one SM may hold
  size_t pair_words = 0;
  if (paired) {
    int per_sm = 0, reserved = 0;
    CU(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CU(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const size_t each = (size_t)per_sm / 2u > (size_t)reserved ? (size_t)per_sm / 2u - (size_t)reserved : 0u;
    pair_words = each > kStaticSmem + 4u * list_words ? (each - kStaticSmem) / 4u - list_words : 0u;
  }
  const uint32_t L = h->L;
  const uint32_t seg_override = prm ? prm->plan_seg_sites : 0;
  h->tau = (prm && prm->plan_tau) ? prm->plan_tau : 128u;
  if (h->tau == 0u) return fail(PCPD_EINVAL, "plan_tau must be positive");
  // Segment tiles below this many core sites cost more in halo windows than they give.
  constexpr uint32_t kMinCore = 4096u;
  bool ring = seg_override == 0 && L <= (batch ? pair_words : avail_words);
  if (paired && !batch && ring && h->G < (uint32_t)sms) {
    // fewer whole columns than SMs would leave SMs idle: cut the columns into segments
    // instead, when two segments of a useful length fit
    const uint32_t tau = (prm && prm->plan_tau) ? prm->plan_tau : 64u;
    const uint64_t halo = (uint64_t)(h->W - 1u) * tau + h->W + 1u;
    if ((uint64_t)L >= 2u * (kMinCore + 2u * halo)) ring = false;
  }
  if (ring) {
    h->ring = true;
    h->core = L;
    h->halo = 0;
    h->n_seg = 1;
    // columns per tile: up to 4 (one phase group), while they fit, the CTA lacks windows and
    // there are still enough tiles to give every SM one
    uint32_t gpi = 1;
    while (gpi < 4 && h->G % (2 * gpi) == 0 && (size_t)(2 * gpi) * L <= (batch ? pair_words : avail_words) &&
           gpi * h->K < 4096 && h->G / (2 * gpi) >= (uint32_t)sms)
      gpi *= 2;
    h->gpi = gpi;
    // a RING tile keeps its columns for a long stretch of sub-steps
    h->tau = (prm && prm->plan_tau) ? prm->plan_tau : (1u << 20);
    uint32_t want = (gpi * h->K + 31u) / 32u * 32u;
    const uint32_t cap = batch ? 256u : pcpdk::kSweepThreads;
    if (want > cap) want = cap;
    if (want < 64u) want = 64u;
    h->threads = want;
    h->tile_words = (size_t)gpi * L;
  } else {
    h->ring = false;
    h->gpi = 1;
    if (paired && !(prm && prm->plan_tau)) h->tau = 64u;
    // W-1 sites per sub-step, + one valid site past the core (pair records), + margin
    h->halo = (h->W - 1u) * h->tau + h->W + 1u;
    uint32_t core;
    if (seg_override) {
      core = seg_override;
    } else {
      const size_t budget = paired ? pair_words : avail_words;
      const size_t max_core = budget > 2u * h->halo ? budget - 2u * h->halo : 0;
      if (max_core < 1024) {
        if (paired) return make_plan(h, prm, kPlanOne);
        return fail(PCPD_EINVAL, "temporal block tau=%u too large for shared memory", h->tau);
      }
      uint32_t nseg = std::max<uint32_t>(2u, (uint32_t)((L + max_core - 1) / max_core));
      if (paired && !batch) {
        // enough tiles per epoch for the two CTAs of every SM, while tiles stay long
        while ((uint64_t)h->G * nseg < 2ull * (uint64_t)sms && (L + nseg) / (nseg + 1u) >= kMinCore) ++nseg;
      }
      for (;; ++nseg) {
        core = (L + nseg - 1) / nseg;
        core = (core + 3u) & ~3u;   // keep tile starts 16-byte aligned
        if (core <= max_core) break;   // the rounding may push a tile past the budget
      }
    }
    // A tile's halo may only reach into its two neighbours (the epoch flags it waits on), so
    // every tile's core, the ragged last one included, must be at least a halo long.  Where the
    // requested length leaves a short last tile, the tiles are evened out (same count, each at
    // most the requested length, starts still 16-byte aligned).
    uint32_t nseg_c = (L + core - 1) / core;
    if (nseg_c >= 2 && L - (nseg_c - 1) * core < h->halo) {
      const uint32_t even = (((L + nseg_c - 1) / nseg_c) + 3u) & ~3u;
      if (even <= core) core = even;
      nseg_c = (L + core - 1) / core;
    }
    if (nseg_c >= 2 && (core < h->halo || L - (nseg_c - 1) * core < h->halo))
      return fail(PCPD_EINVAL, "segment tiles of %u sites (last %u) are shorter than the halo of %u sites", core,
                  L - (nseg_c - 1) * core, h->halo);
    h->core = core;
    h->n_seg = nseg_c;
    h->tile_words = (size_t)core + 2u * h->halo;
    if (h->tile_words > avail_words) return fail(PCPD_EINVAL, "tile of %zu sites exceeds shared memory", h->tile_words);
    // a tile shorter than L - 4W sees fewer candidate windows than the ring has
    if (h->n_seg < 2 || h->tile_words + 4u * h->W > L)
      return fail(PCPD_EINVAL, "segmented plan needs >= 2 tiles each shorter than L-4W (L=%u, core=%u, halo=%u)", L, core, h->halo);
    h->threads = paired ? 256u : pcpdk::kSweepThreads;
  }
  if (prm && prm->plan_threads) {
    if (prm->plan_threads % 32 || prm->plan_threads > pcpdk::kSweepThreads || prm->plan_threads < 64)
      return fail(PCPD_EINVAL, "plan_threads must be a multiple of 32 in [64, %u]", pcpdk::kSweepThreads);
    h->threads = prm->plan_threads;
  }
  h->dyn_smem = 4 * (h->tile_words + list_words);
  rc = raise_smem_limit();
  if (rc) return rc;
  int per_sm = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel(false, h->W), (int)h->threads, h->dyn_smem));
  if (paired && (batch || !h->ring) && per_sm < 2) return make_plan(h, prm, kPlanOne);   // the pair does not fit
  if (per_sm < 1) return fail(PCPD_EINVAL, "tile plan does not fit one CTA per SM");
  h->grid = per_sm * sms;
  const uint64_t tiles = (uint64_t)(h->G / h->gpi) * h->n_seg;
  if (paired && !h->ring && tiles >= (1ull << 24)) return make_plan(h, prm, kPlanOne);   // longer tiles
  if (tiles >= (1ull << 24))   // a work item carries the tile index in 24 bits
    return fail(PCPD_EINVAL, "%llu tiles per epoch (at most 2^24 - 1): fewer samples or longer tiles",
                (unsigned long long)tiles);
  h->tiles = (uint32_t)tiles;
  return PCPD_OK;
}

// Device buffers allocated for a handle but not yet handed to it: freed on an early return
// (an error), so that the handle keeps its old buffers and nothing leaks.
struct FreeUnlessKept {
  void **p[3];
  bool keep = false;
  ~FreeUnlessKept() {
    if (keep) return;
    for (void **q : p)
      if (q && *q) cudaFree(*q);
  }
};

int ensure_records(pcpd_t *h, size_t need) {
  if (need <= h->rec_cap) return PCPD_OK;
  size_t cap = h->rec_cap ? h->rec_cap : 64;
  while (cap < need) cap *= 2;
  unsigned long long *nt = nullptr, *np = nullptr;
  uint32_t *ns = nullptr;
  FreeUnlessKept pending{{(void **)&nt, (void **)&np, (void **)&ns}};
  int rc = dev_alloc((void **)&nt, cap * sizeof(unsigned long long), "record totals");
  if (!rc) rc = dev_alloc((void **)&np, cap * sizeof(unsigned long long), "record pair counts");
  if (!rc && h->per_sample) rc = dev_alloc((void **)&ns, cap * (size_t)h->S * sizeof(uint32_t), "per-sample records");
  if (rc) return rc;
  CU(cudaMemsetAsync(nt, 0, cap * sizeof(unsigned long long), h->stream));
  CU(cudaMemsetAsync(np, 0, cap * sizeof(unsigned long long), h->stream));
  if (h->per_sample) CU(cudaMemsetAsync(ns, 0, cap * (size_t)h->S * sizeof(uint32_t), h->stream));
  const size_t have = h->rec_times.size();
  if (have) {
    CU(cudaMemcpyAsync(nt, h->d_rec_total, have * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemcpyAsync(np, h->d_rec_pairs, have * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream));
    if (h->per_sample)
      CU(cudaMemcpyAsync(ns, h->d_rec_sample, have * (size_t)h->S * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream));
  }
  CU(cudaStreamSynchronize(h->stream));
  pending.keep = true;
  cudaFree(h->d_rec_total);
  cudaFree(h->d_rec_pairs);
  cudaFree(h->d_rec_sample);
  h->d_rec_total = nt;
  h->d_rec_pairs = np;
  h->d_rec_sample = ns;
  h->rec_cap = cap;
  return PCPD_OK;
}

int ensure_rec_sub(pcpd_t *h, size_t need) {
  if (need <= h->rec_sub_cap) return PCPD_OK;
  size_t cap = h->rec_sub_cap ? h->rec_sub_cap : 64;
  while (cap < need) cap *= 2;
  CU(cudaStreamSynchronize(h->stream));
  cudaFree(h->d_rec_sub);
  h->d_rec_sub = nullptr;
  h->rec_sub_cap = 0;   // no buffer until the new one exists
  const int rc = dev_alloc((void **)&h->d_rec_sub, cap * sizeof(uint32_t), "record sub-steps");
  if (rc) return rc;
  h->rec_sub_cap = cap;
  return PCPD_OK;
}

// Descriptor of handle h for sub-steps [n_begin, n_end), records subs[ri..rj) in slots from slot.
void fill_desc(const pcpd_t *h, pcpdk::InstDesc &D, uint64_t n_begin, uint64_t n_end, size_t ri, size_t rj,
               size_t slot) {
  memset(&D, 0, sizeof D);
  D.L = h->L;
  D.K = h->K;
  D.W = h->W;
  D.g_base = h->g_base;
  D.G = h->G;
  D.S = h->S;
  D.pitch = h->pitch;
  D.k0 = h->k0;
  D.k1 = h->k1;
  D.ring = h->ring ? 1u : 0u;
  D.gpi = h->gpi;
  D.core = h->core;
  D.halo = h->halo;
  D.tau = h->tau;
  D.n_seg = h->n_seg;
  D.n_begin = (uint32_t)n_begin;
  D.n_end = (uint32_t)n_end;
  D.n_rec = (uint32_t)(rj - ri);
  D.buf0 = h->buf[h->cur];
  D.buf1 = h->buf[1 - h->cur];
  D.rec_sub = h->d_rec_sub ? h->d_rec_sub + ri : nullptr;
  D.rec_total = h->d_rec_total ? h->d_rec_total + slot : nullptr;
  D.rec_sample = h->per_sample ? h->d_rec_sample + slot * (size_t)h->S : nullptr;
  D.rec_pairs = h->d_rec_pairs ? h->d_rec_pairs + slot : nullptr;
  D.done = h->d_done;
  D.rk = pcpdk::make_round_keys(h->k0, h->k1);
  D.T = h->T;
}

int tuned_plan(const pcpd_params *prm, pcpd_params *out);

// The error word of the engine: 0, or a device-side wait that ran out of its budget.
int check_engine(const pcpd_t *h) {
  uint32_t err = 0;
  CU(cudaMemcpyAsync(&err, h->d_done + h->tiles + 1, 4, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  if (err) return fail(PCPD_ETIMEOUT, "device wait ran out of its budget (code %u)", err);
  return PCPD_OK;
}

// Clock cycles an engine item may wait for another item or a copy before it gives up.
constexpr unsigned long long kSpinLimit = 40ull * 1000 * 1000 * 1000;   // ~20 s at 2 GHz

// Sweep from n_now to n_end in engine launches; records subs[0..) (absolute sub-steps in
// (n_now, n_end], already copied to d_rec_sub) go to record slots [slot0, ...).
int launch_sweep(pcpd_t *h, uint64_t n_end, const std::vector<uint64_t> &subs, size_t slot0) {
  // epochs per launch: the epoch field of a work item has 24 bits, and the launch's item
  // count (epochs x tiles) must fit 32 bits
  const uint64_t max_epochs = std::min<uint64_t>(1u << 22, 0xFFFFFFFFull / h->tiles);
  size_t ri = 0;
  while (h->n_now < n_end) {
    const uint64_t span = n_end - h->n_now;
    const uint64_t epochs_all = (span + h->tau - 1) / h->tau;
    const uint64_t epochs = epochs_all > max_epochs ? max_epochs : epochs_all;
    const uint64_t nb = (epochs == epochs_all) ? n_end : h->n_now + epochs * h->tau;
    size_t rj = ri;
    while (rj < subs.size() && subs[rj] <= nb) ++rj;
    pcpdk::BatchParams B;
    memset(&B, 0, sizeof B);
    pcpdk::InstDesc &D = B.single;
    D.L = h->L;
    D.K = h->K;
    D.W = h->W;
    D.g_base = h->g_base;
    D.G = h->G;
    D.S = h->S;
    D.pitch = h->pitch;
    D.k0 = h->k0;
    D.k1 = h->k1;
    D.ring = h->ring ? 1u : 0u;
    D.gpi = h->gpi;
    D.core = h->core;
    D.halo = h->halo;
    D.tau = h->tau;
    D.n_seg = h->n_seg;
    D.n_begin = (uint32_t)h->n_now;
    D.n_end = (uint32_t)nb;
    D.n_rec = (uint32_t)(rj - ri);
    D.buf0 = h->buf[h->cur];
    D.buf1 = h->buf[1 - h->cur];
    D.rec_sub = h->d_rec_sub + ri;
    D.rec_total = h->d_rec_total ? h->d_rec_total + slot0 + ri : nullptr;
    D.rec_sample = h->per_sample ? h->d_rec_sample + (slot0 + ri) * (size_t)h->S : nullptr;
    D.rec_pairs = h->d_rec_pairs ? h->d_rec_pairs + slot0 + ri : nullptr;
    D.done = h->d_done;
    D.rk = pcpdk::make_round_keys(h->k0, h->k1);
    D.T = h->T;
    CU(cudaMemsetAsync(h->d_done, 0, (h->tiles + 1) * sizeof(uint32_t), h->stream));  // flags + counter
    B.items = nullptr;
    B.n_items = (uint32_t)(epochs * h->tiles);
    B.tiles_per_epoch = h->tiles;
    B.counter = h->d_done + h->tiles;
    B.err = h->d_done + h->tiles + 1;
    B.tile_words = (uint32_t)h->tile_words;
    B.spin_limit = kSpinLimit;
    const int grid = (int)((uint64_t)h->grid < B.n_items ? (uint64_t)h->grid : B.n_items);
    if (h->jit_fn) {
      void *args[] = {&B};
      const CUresult r = g_jit_api.launch(h->jit_fn, grid, 1, 1, h->threads, 1, 1, (unsigned)h->dyn_smem,
                                          (CUstream)h->stream, args, nullptr);
      if (r != CUDA_SUCCESS) return fail(PCPD_ECUDA, "launch of the runtime-compiled sweep failed (%d)", (int)r);
    } else {
      sweep_kernel(false, h->W)<<<grid, h->threads, h->dyn_smem, h->stream>>>(B);
      CU(cudaGetLastError());
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (epochs & 1u) h->cur = 1 - h->cur;
    h->n_now = nb;
    ri = rj;
  }
  return PCPD_OK;
}

}  // namespace

extern "C" {

const char *pcpd_last_error(void) { return g_err.c_str(); }

int pcpd_debug_build(void) {
#ifdef PCPD_DEBUG
  return 1;
#else
  return 0;
#endif
}

unsigned int pcpd_debug_check(void) {
#ifdef PCPD_DEBUG
  unsigned int v = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return ~0u;
  if (cudaMemcpyFromSymbol(&v, pcpdk::g_debug_err, sizeof v) != cudaSuccess) return ~0u;
  if (cudaMemcpyToSymbol(pcpdk::g_debug_err, &zero, sizeof zero) != cudaSuccess) return ~0u;
  return v;
#else
  return 0u;
#endif
}

unsigned long long pcpd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int pcpd_thresholds(double p, double d, uint64_t *t_d, uint64_t *t_da) {
  if (!t_d || !t_da) return fail(PCPD_EINVAL, "NULL output");
  return thresholds(p, d, t_d, t_da);
}

uint64_t pcpd_substep_of_time(uint32_t L, uint64_t t) { return L < 3 ? 0 : substep_of_time(L, t); }

uint64_t pcpd_substep_of_time_n(uint32_t L, uint32_t tuple, uint64_t t) {
  const uint32_t W = (tuple ? tuple : 2u) + 1u;
  return (tuple == 1u || tuple > 4u || L < W) ? 0 : substep_of_time(L, t, W);
}

}  // extern "C"

namespace {

// A handle; BATCH_MEMBER: it runs in batched launches (one CTA shape for every instance of a
// launch), so its SEGMENT tiles take the one-CTA-per-SM plan.
int create_handle(const pcpd_params *prm, pcpd_t **out, bool batch_member) {
  if (!prm || !out) return fail(PCPD_EINVAL, "NULL argument");
  *out = nullptr;
  if (prm->L < 3 || prm->L >= (1u << 30)) return fail(PCPD_EINVAL, "L must satisfy 3 <= L < 2^30 (L=%u)", prm->L);
  if (prm->samples == 0 || prm->samples % 32 || prm->samples > (1u << 22))
    return fail(PCPD_EINVAL, "samples must be a positive multiple of 32, at most 2^22 (samples=%u)", prm->samples);
  if (prm->init < 0 || prm->init > 2) return fail(PCPD_EINVAL, "unknown init mode %d", prm->init);
  if (prm->tuple == 1u || prm->tuple > 4u) return fail(PCPD_EINVAL, "tuple must be 0 or 2 (PCPD), 3 (TCPD) or 4 (QCPD) (tuple=%u)", prm->tuple);
  if (prm->L < (prm->tuple ? prm->tuple : 2u) + 1u) return fail(PCPD_EINVAL, "L=%u is shorter than one window", prm->L);
  if (prm->group0 % 4u || (uint64_t)prm->group0 + prm->samples / 32u > (1ull << 26))
    return fail(PCPD_EINVAL, "group0 must be a multiple of 4 with group0 + samples/32 <= 2^26 (group0=%u)", prm->group0);
  uint64_t td, tda;
  int rc = thresholds(prm->p, prm->d, &td, &tda);
  if (rc) return rc;
  rc = device_check();
  if (rc) return rc;

  pcpd_params tuned;
  if (prm->autotune && !prm->plan_threads && !prm->plan_seg_sites && !prm->plan_tau) {
    rc = tuned_plan(prm, &tuned);
    if (rc) return rc;
    prm = &tuned;
  }
  pcpd_t *h = new pcpd();
  h->L = prm->L;
  h->W = (prm->tuple ? prm->tuple : 2u) + 1u;
  h->g_base = prm->group0;
  h->K = prm->L / h->W;
  h->S = prm->samples;
  h->G = prm->samples / 32u;
  h->p = prm->p;
  h->d = prm->d;
  h->seed = prm->seed;
  h->td = td;
  h->tda = tda;
  h->T = split_thresholds(td, tda);
  h->k0 = (uint32_t)(prm->seed & 0xFFFFFFFFu);
  h->k1 = (uint32_t)(prm->seed >> 32);
  h->init = prm->init;
  h->per_sample = prm->per_sample != 0;
  auto bail = [&](int code) {
    pcpd_destroy(h);
    return code;
  };
  rc = make_plan(h, prm, batch_member ? kPlanPairedBatch : kPlanPaired);
  if (rc) return bail(rc);
  if (prm->stream) {
    h->stream = (cudaStream_t)prm->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(PCPD_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    h->own_stream = true;
  }
  // device rows are padded to a multiple of 4 words so that tiles can move by TMA
  h->pitch = (h->L + 3u) & ~3u;
  const size_t words = (size_t)h->G * h->pitch;
  if (prm->dev_lattice) {
    if (prm->dev_bytes < 2 * words * 4 || ((uintptr_t)prm->dev_lattice & 255u))
      return bail(fail(PCPD_EINVAL, "dev_lattice must be 256-byte aligned and hold 2*G*ceil4(L) words (%zu bytes)", 2 * words * 4));
    h->buf[0] = (uint32_t *)prm->dev_lattice;
    h->buf[1] = h->buf[0] + words;
  } else {
    const int ra = dev_alloc((void **)&h->buf[0], 2 * words * 4, "lattice");
    if (ra) return bail(ra);
    h->buf[1] = h->buf[0] + words;
    h->own_mem = true;
  }
  {
    cudaError_t e = cudaMalloc(&h->d_done, (h->tiles + 2) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_done, 0, (h->tiles + 2) * sizeof(uint32_t), h->stream);
    if (e != cudaSuccess) return bail(fail(PCPD_ENOMEM, "engine scratch: %s", cudaGetErrorString(e)));
  }
  pcpdk::k_init<<<1024, 256, 0, h->stream>>>(h->buf[0], h->L, h->pitch, h->G, h->init, h->k0, h->k1, h->g_base);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bail(fail(PCPD_ECUDA, "init launch: %s", cudaGetErrorString(e)));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  // specialised sweep: thresholds strictly inside (0, 2^32) only
  const bool normal = !h->T.td_full && !h->T.tda_full && h->T.td != 0u && h->T.tda != 0u;
  const bool want = prm->jit > 0 || (prm->jit == 0 && (uint64_t)h->G * h->L >= (1ull << 22));
  if (normal && want) {
    CUfunction fn = nullptr;
    if (jit_function(h->T.td, h->T.tda, h->W, &fn) == PCPD_OK) {
      int per_sm = 0, sms = 0, dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (g_jit_api.occupancy(&per_sm, fn, (int)h->threads, h->dyn_smem) == CUDA_SUCCESS &&
          per_sm >= 1) {
        h->jit_fn = fn;
        h->grid = per_sm * sms;
      }
    } else if (prm->jit > 0) {
      return bail(PCPD_ECUDA);   // asked for explicitly: report why
    }
    g_err.clear();
  }
  *out = h;
  return PCPD_OK;
}

}  // namespace

extern "C" {

int pcpd_create_ex(const pcpd_params *prm, pcpd_t **out) { return create_handle(prm, out, false); }

pcpd_t *pcpd_create(uint32_t L, uint32_t samples, double p, double d, uint64_t seed) {
  pcpd_params prm;
  memset(&prm, 0, sizeof prm);
  prm.L = L;
  prm.samples = samples;
  prm.p = p;
  prm.d = d;
  prm.seed = seed;
  pcpd_t *h = nullptr;
  return pcpd_create_ex(&prm, &h) == PCPD_OK ? h : nullptr;
}

void pcpd_destroy(pcpd_t *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_mem) cudaFree(h->buf[0]);
  cudaFree(h->d_done);
  cudaFree(h->d_rec_total);
  cudaFree(h->d_rec_pairs);
  cudaFree(h->d_rec_sample);
  cudaFree(h->d_rec_sub);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

int pcpd_run(pcpd_t *h, uint64_t steps_mcs, const uint64_t *times, size_t n_times) {
  NvtxRange nvtx("pcpd_run");
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  if (n_times && !times) return fail(PCPD_EINVAL, "record_times_mcs is NULL");
  const uint64_t t_end = h->t_now + steps_mcs;
  if (t_end < h->t_now) return fail(PCPD_EINVAL, "time overflow");
  const uint64_t n_end = steps_mcs ? substep_of_time(h->L, t_end, h->W) : h->n_now;
  if (n_end > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "sub-step count %llu would reach 2^32", (unsigned long long)n_end);
  bool now_first = false;
  std::vector<uint64_t> subs;
  for (size_t i = 0; i < n_times; ++i) {
    const uint64_t t = times[i];
    if (i && t <= times[i - 1]) return fail(PCPD_EINVAL, "record times must be strictly increasing");
    if (t == h->t_now && i == 0 && h->n_now == substep_of_time(h->L, t, h->W)) {
      now_first = true;
      continue;
    }
    if (t <= h->t_now || t > t_end)
      return fail(PCPD_EINVAL, "record time %llu outside (%llu, %llu]", (unsigned long long)t,
                  (unsigned long long)h->t_now, (unsigned long long)t_end);
    subs.push_back(substep_of_time(h->L, t, h->W));
  }
  const size_t slot0 = h->rec_times.size();
  int rc = ensure_records(h, slot0 + n_times);
  if (rc) return rc;
  size_t slot = slot0;
  if (now_first) {
    pcpdk::k_count<<<h->G, 256, 0, h->stream>>>(h->buf[h->cur], h->L, h->pitch, h->S, h->d_rec_total + slot,
                                                 h->per_sample ? h->d_rec_sample + slot * (size_t)h->S : nullptr,
                                                 h->d_rec_pairs + slot);
    CU(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++slot;
  }
  if (!subs.empty()) {
    rc = ensure_rec_sub(h, subs.size());
    if (rc) return rc;
    std::vector<uint32_t> s32(subs.begin(), subs.end());
    CU(cudaMemcpyAsync(h->d_rec_sub, s32.data(), s32.size() * 4, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));  // s32 is a local buffer
  }
  rc = launch_sweep(h, n_end, subs, slot);
  if (rc) return rc;
  for (size_t i = 0; i < n_times; ++i) h->rec_times.push_back(times[i]);
  h->t_now = t_end;
  return PCPD_OK;
}

int pcpd_run_substeps(pcpd_t *h, uint64_t n_substeps) {
  NvtxRange nvtx("pcpd_run_substeps");
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  const uint64_t n_end = h->n_now + n_substeps;
  if (n_end > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "sub-step count would reach 2^32");
  std::vector<uint64_t> none;
  int rc = launch_sweep(h, n_end, none, h->rec_times.size());
  if (rc) return rc;
  h->t_now = time_of_substep(h->L, h->n_now, h->W);
  return PCPD_OK;
}

size_t pcpd_num_records(const pcpd_t *h) { return h ? h->rec_times.size() : 0; }

int pcpd_get_plan(const pcpd_t *h, pcpd_plan_info *out) {
  if (!h || !out) return fail(PCPD_EINVAL, "NULL argument");
  memset(out, 0, sizeof *out);
  out->ring = h->ring ? 1u : 0u;
  out->gpi = h->gpi;
  out->threads = h->threads;
  out->core = h->core;
  out->halo = h->halo;
  out->tau = h->tau;
  out->n_seg = h->n_seg;
  out->tiles = h->tiles;
  out->grid = (uint32_t)h->grid;
  out->jit = h->jit_fn ? 1u : 0u;
  out->smem_bytes = h->dyn_smem;
  return PCPD_OK;
}

uint64_t pcpd_substep(const pcpd_t *h) { return h ? h->n_now : 0; }
uint64_t pcpd_time_mcs(const pcpd_t *h) { return h ? h->t_now : 0; }

int pcpd_sync(pcpd_t *h) {
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  CU(cudaStreamSynchronize(h->stream));
  return check_engine(h);
}

int pcpd_density(const pcpd_t *h, double *rho_out, uint64_t *counts_out, size_t n) {
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  if (n > h->rec_times.size()) return fail(PCPD_EINVAL, "only %zu records", h->rec_times.size());
  if (n == 0) return PCPD_OK;
  std::vector<unsigned long long> c(n);
  CU(cudaMemcpyAsync(c.data(), h->d_rec_total, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  int rc = check_engine(h);
  if (rc) return rc;
  const double denom = (double)h->L * (double)h->S;
  for (size_t i = 0; i < n; ++i) {
    if (counts_out) counts_out[i] = c[i];
    if (rho_out) rho_out[i] = (double)c[i] / denom;
  }
  return PCPD_OK;
}

int pcpd_record_times(const pcpd_t *h, uint64_t *times_out, size_t n) {
  if (!h || !times_out) return fail(PCPD_EINVAL, "NULL argument");
  if (n > h->rec_times.size()) return fail(PCPD_EINVAL, "only %zu records", h->rec_times.size());
  for (size_t i = 0; i < n; ++i) times_out[i] = h->rec_times[i];
  return PCPD_OK;
}

int pcpd_pair_counts(const pcpd_t *h, uint64_t *counts_out, size_t n) {
  if (!h || (n && !counts_out)) return fail(PCPD_EINVAL, "NULL argument");
  if (n > h->rec_times.size()) return fail(PCPD_EINVAL, "only %zu records", h->rec_times.size());
  if (n == 0) return PCPD_OK;
  std::vector<unsigned long long> c(n);
  CU(cudaMemcpyAsync(c.data(), h->d_rec_pairs, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  int rc = check_engine(h);
  if (rc) return rc;
  for (size_t i = 0; i < n; ++i) counts_out[i] = c[i];
  return PCPD_OK;
}

int pcpd_pair_density(const pcpd_t *h, double *rho_pair_out, size_t n) {
  if (!h || (n && !rho_pair_out)) return fail(PCPD_EINVAL, "NULL argument");
  std::vector<uint64_t> c(n);
  const int rc = pcpd_pair_counts(h, c.data(), n);
  if (rc) return rc;
  const double norm = (double)h->L * (double)h->S;
  for (size_t i = 0; i < n; ++i) rho_pair_out[i] = (double)c[i] / norm;
  return PCPD_OK;
}

int pcpd_sample_counts(const pcpd_t *h, size_t r, uint32_t *out) {
  if (!h || !out) return fail(PCPD_EINVAL, "NULL argument");
  if (!h->per_sample) return fail(PCPD_ESTATE, "per-sample counts were not requested at creation");
  if (r >= h->rec_times.size()) return fail(PCPD_EINVAL, "record %zu does not exist", r);
  CU(cudaMemcpyAsync(out, h->d_rec_sample + r * (size_t)h->S, (size_t)h->S * 4, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return PCPD_OK;
}

namespace {

int get_lattice(const pcpd_t *h, uint32_t *host_out, bool wait) {
  if (!h || !host_out) return fail(PCPD_EINVAL, "NULL argument");
  CU(cudaMemcpy2DAsync(host_out, (size_t)h->L * 4, h->buf[h->cur], (size_t)h->pitch * 4, (size_t)h->L * 4, h->G,
                       cudaMemcpyDeviceToHost, h->stream));
  if (!wait) return PCPD_OK;
  CU(cudaStreamSynchronize(h->stream));
  return check_engine(h);
}

int set_lattice(pcpd_t *h, const uint32_t *host_in, uint64_t substep, bool wait) {
  if (!h || !host_in) return fail(PCPD_EINVAL, "NULL argument");
  if (substep > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "sub-step must be < 2^32");
  CU(cudaMemcpy2DAsync(h->buf[h->cur], (size_t)h->pitch * 4, host_in, (size_t)h->L * 4, (size_t)h->L * 4, h->G,
                       cudaMemcpyHostToDevice, h->stream));
  if (wait) CU(cudaStreamSynchronize(h->stream));
  h->n_now = substep;
  h->t_now = time_of_substep(h->L, substep, h->W);
  h->rec_times.clear();
  if (h->d_rec_total) CU(cudaMemsetAsync(h->d_rec_total, 0, h->rec_cap * sizeof(unsigned long long), h->stream));
  if (h->d_rec_pairs) CU(cudaMemsetAsync(h->d_rec_pairs, 0, h->rec_cap * sizeof(unsigned long long), h->stream));
  if (h->d_rec_sample) CU(cudaMemsetAsync(h->d_rec_sample, 0, h->rec_cap * (size_t)h->S * 4, h->stream));
  return PCPD_OK;
}

}  // namespace

int pcpd_get_lattice(const pcpd_t *h, uint32_t *host_out) { return get_lattice(h, host_out, true); }

int pcpd_get_lattice_async(const pcpd_t *h, uint32_t *host_out) { return get_lattice(h, host_out, false); }

int pcpd_set_lattice(pcpd_t *h, const uint32_t *host_in, uint64_t substep) {
  return set_lattice(h, host_in, substep, true);
}

int pcpd_set_lattice_async(pcpd_t *h, const uint32_t *host_in, uint64_t substep) {
  return set_lattice(h, host_in, substep, false);
}

int pcpd_dev_philox(const uint32_t *ctr, uint64_t seed, uint32_t *out, size_t n, void *stream) {
  int rc = device_check();
  if (rc) return rc;
  if (n == 0) return PCPD_OK;
  if (!ctr || !out) return fail(PCPD_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  pcpdk::k_philox<<<256, 256, 0, s>>>(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), out, n);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return PCPD_OK;
}

int pcpd_dev_rate_masks(const uint32_t *words, uint64_t t_d, uint64_t t_da, uint32_t *masks,
                        size_t n, void *stream) {
  int rc = device_check();
  if (rc) return rc;
  if (n == 0) return PCPD_OK;
  if (!words || !masks) return fail(PCPD_EINVAL, "NULL argument");
  if (t_d > kTwo32 || t_da > kTwo32 || t_d > t_da) return fail(PCPD_EINVAL, "need T_D <= T_DA <= 2^32");
  cudaStream_t s = (cudaStream_t)stream;
  pcpdk::k_rate_masks<<<256, 256, 0, s>>>(words, split_thresholds(t_d, t_da), masks, n);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return PCPD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free sweep (pcpd_sweep_noalloc).  Its scratch -- per-tile epoch flags, the work
// counter and the error word -- lives in this fixed device array instead of memory the
// library allocates.  The array exists on every device that loads the library, until exit.
// ------------------------------------------------------------------------------------------
namespace {

constexpr uint32_t kNoAllocMaxTiles = 16384;   // tiles per epoch the array can serve
constexpr size_t kNoAllocScratchWords = kNoAllocMaxTiles + 64;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchWords];

// Device address of the scratch array on the current device.  In host code the array's name
// is only a host-side stand-in; the address is looked up on every call (cheap, allocates
// nothing), so a context re-created after cudaDeviceReset gets its own.
int noalloc_scratch(uint32_t **out) {
  int dev = 0;
  CU(cudaGetDevice(&dev));
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(PCPD_ECUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
  *out = (uint32_t *)p;
  return PCPD_OK;
}

}  // namespace

extern "C" int pcpd_sweep_noalloc(uint32_t *lat_in, uint32_t *lat_out, uint32_t L, uint32_t samples,
                                  double p, double d, uint64_t seed, uint64_t substep_begin,
                                  uint64_t n_substeps, void *stream) {
  if (!lat_in || !lat_out || lat_in == lat_out) return fail(PCPD_EINVAL, "need two distinct device lattices");
  if (L < 3 || L >= (1u << 30)) return fail(PCPD_EINVAL, "L must satisfy 3 <= L < 2^30 (L=%u)", L);
  if (samples == 0 || samples % 32 || samples > (1u << 22))
    return fail(PCPD_EINVAL, "samples must be a positive multiple of 32, at most 2^22 (samples=%u)", samples);
  if (substep_begin + n_substeps > 0xFFFFFFFFull || substep_begin + n_substeps < substep_begin)
    return fail(PCPD_EINVAL, "sub-step count would reach 2^32");
  uint64_t td, tda;
  int rc = thresholds(p, d, &td, &tda);
  if (rc) return rc;
  rc = device_check();
  if (rc) return rc;
  pcpd h;   // plan only: no device memory is attached to it
  h.L = L;
  h.K = L / 3u;
  h.S = samples;
  h.G = samples / 32u;
  h.pitch = L;
  h.T = split_thresholds(td, tda);
  h.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  h.k1 = (uint32_t)(seed >> 32);
  rc = make_plan(&h, nullptr);
  if (rc) return rc;
  if (h.tiles > kNoAllocMaxTiles)
    return fail(PCPD_EINVAL, "%u tiles per epoch exceed the %u the allocation-free scratch holds (L=%u, samples=%u)",
                h.tiles, kNoAllocMaxTiles, L, samples);
  const size_t bytes = (size_t)(samples / 32u) * L * 4u;
  if ((((uintptr_t)lat_in | (uintptr_t)lat_out) & 3u) != 0u)
    return fail(PCPD_EINVAL, "lattice pointers must be 4-byte aligned");
  if ((const char *)lat_in < (const char *)lat_out + bytes && (const char *)lat_out < (const char *)lat_in + bytes)
    return fail(PCPD_EINVAL, "lat_in and lat_out overlap");
  uint32_t *scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  uint32_t *bufs[2] = {lat_in, lat_out};
  int cur = 0;
  uint64_t n_now = substep_begin;
  const uint64_t n_end = substep_begin + n_substeps;
  const uint64_t max_epochs = std::min<uint64_t>(1u << 22, 0xFFFFFFFFull / h.tiles);
  while (n_now < n_end) {
    const uint64_t span = n_end - n_now;
    const uint64_t epochs_all = (span + h.tau - 1) / h.tau;
    const uint64_t epochs = epochs_all > max_epochs ? max_epochs : epochs_all;
    const uint64_t nb = (epochs == epochs_all) ? n_end : n_now + epochs * h.tau;
    pcpdk::BatchParams B;
    memset(&B, 0, sizeof B);
    pcpdk::InstDesc &D = B.single;
    D.L = L;
    D.K = h.K;
    D.W = h.W;
    D.G = h.G;
    D.S = samples;
    D.pitch = L;
    D.k0 = h.k0;
    D.k1 = h.k1;
    D.ring = h.ring ? 1u : 0u;
    D.gpi = h.gpi;
    D.core = h.core;
    D.halo = h.halo;
    D.tau = h.tau;
    D.n_seg = h.n_seg;
    D.n_begin = (uint32_t)n_now;
    D.n_end = (uint32_t)nb;
    D.buf0 = bufs[cur];
    D.buf1 = bufs[1 - cur];
    D.done = scratch;
    D.rk = pcpdk::make_round_keys(h.k0, h.k1);
    D.T = h.T;
    // every call starts from cleared flags, counter and error word
    CU(cudaMemsetAsync(scratch, 0, (h.tiles + 2) * sizeof(uint32_t), s));
    B.items = nullptr;
    B.n_items = (uint32_t)(epochs * h.tiles);
    B.tiles_per_epoch = h.tiles;
    B.counter = scratch + h.tiles;
    B.err = scratch + h.tiles + 1;
    B.tile_words = (uint32_t)h.tile_words;
    B.spin_limit = kSpinLimit;
    const int grid = (int)((uint64_t)h.grid < B.n_items ? (uint64_t)h.grid : B.n_items);
    sweep_kernel(false, 3u)<<<grid, h.threads, h.dyn_smem, s>>>(B);
    CU(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    uint32_t err = 0;
    CU(cudaMemcpyAsync(&err, scratch + h.tiles + 1, 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (err) return fail(PCPD_ETIMEOUT, "device wait ran out of its budget (code %u)", err);
    if (epochs & 1u) cur = 1 - cur;
    n_now = nb;
  }
  // the result must end in lat_out
  if (cur == 0) {
    CU(cudaMemcpyAsync(lat_out, lat_in, bytes, cudaMemcpyDeviceToDevice, s));
    CU(cudaStreamSynchronize(s));
  }
  return PCPD_OK;
}

// ------------------------------------------------------------------------------------------
// Batches: many instances (any L, samples, p, d, seed, step count, records) in one persistent
// launch of the engine over an explicit item list.
// ------------------------------------------------------------------------------------------
namespace {
// A batch round as a CUDA graph: the item-list and descriptor uploads (from pinned staging
// buffers), the counter reset and the engine launch, captured once and updated in place
// (cudaGraphExecUpdate) for later rounds of the same shape.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  unsigned long long *h_items = nullptr;   // pinned
  size_t h_items_cap = 0;
  pcpdk::InstDesc *h_desc = nullptr;       // pinned, kMaxBatchInst entries
  ~GraphCache() {
    if (exec) cudaGraphExecDestroy(exec);
    if (h_items) cudaFreeHost(h_items);
    if (h_desc) cudaFreeHost(h_desc);
  }
};

}  // namespace

struct pcpd_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<pcpd_t *> inst;
  std::vector<uint64_t> steps;
  std::vector<std::vector<uint64_t>> rec;
  unsigned long long *d_items = nullptr;
  size_t items_cap = 0;
  uint32_t *d_ctl = nullptr;   // work counter, error word
  bool ran = false;
  int jit = 0;                 // see pcpd_batch_set_jit
  size_t jit_launches = 0;
  GraphCache gc;
};

namespace {
std::mutex g_batch_mu;   // the constant-memory descriptor table serves one batch launch at a time

// One instance's share of a multi-instance launch: advance h from h->n_now to n_end; its
// record sub-steps are rec_sub (all of them, increasing, already on the device in
// h->d_rec_sub); records rec_first.. that fall in (n_now, n_end] go to slots slot0.. .
struct MultiTarget {
  pcpd_t *h = nullptr;
  uint64_t n_end = 0;
  std::vector<uint64_t> rec_sub;
  size_t rec_first = 0;
  size_t slot0 = 0;
  size_t rec_taken = 0;   // out: records that fell in this launch
};

// Advance every target in engine launches of at most kMaxBatchInst instances each; the item
// list starts every segmented chain at once and spreads the whole-ring items (longest first)
// between its epochs.  Waits for completion; updates each handle's buffer and clock.
// Members of a batch that share a threshold pair and window width whose work reaches this many
// attempted updates run a kernel compiled for that pair (as a lone instance does); below it the
// compile (about 1.5 s, once per process and pair) would cost more than it saves.
constexpr double kJitBatchMinAttempts = 2e13;

// jit_mode: > 0 compile for every pair two or more members share, 0 when their work reaches
// kJitBatchMinAttempts, < 0 never.  *jit_launches (nullable) counts the launches that ran a
// runtime-compiled kernel.
int run_multi(cudaStream_t stream, uint32_t *d_ctl, unsigned long long **d_items, size_t *items_cap,
              std::vector<MultiTarget> &tg, GraphCache &gc, int jit_mode = -1, size_t *jit_launches = nullptr) {
  int dev = 0, sms = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t n = tg.size();
  std::vector<uint64_t> epochs(n);
  for (size_t i = 0; i < n; ++i) {
    pcpd_t *h = tg[i].h;
    if (tg[i].n_end < h->n_now) return fail(PCPD_EINVAL, "target sub-step behind the clock");
    if (tg[i].n_end > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "sub-step count would reach 2^32");
    epochs[i] = (tg[i].n_end - h->n_now + h->tau - 1) / h->tau;
    if (epochs[i] >= (1u << 24)) return fail(PCPD_EINVAL, "instance %zu needs too many epochs", i);
    CU(cudaMemsetAsync(h->d_done, 0, (h->tiles + 2) * sizeof(uint32_t), stream));
    size_t rj = tg[i].rec_first;
    while (rj < tg[i].rec_sub.size() && tg[i].rec_sub[rj] <= tg[i].n_end) ++rj;
    tg[i].rec_taken = rj - tg[i].rec_first;
  }
  // Launch chunks of at most kMaxBatchInst members: first the members that share a threshold
  // pair (and window width) worth a runtime-compiled kernel, one pair per chunk; then the rest,
  // in order, on the generic kernel.  The grouping changes no result bit.
  struct Chunk {
    std::vector<size_t> ids;
    const JitEntry *jit = nullptr;
  };
  std::vector<Chunk> chunks;
  {
    std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<size_t>> groups;
    std::vector<size_t> rest;
    for (size_t i = 0; i < n; ++i) {
      const pcpd_t *h = tg[i].h;
      const bool normal = !h->T.td_full && !h->T.tda_full && h->T.td != 0u && h->T.tda != 0u;
      if (jit_mode >= 0 && normal && epochs[i] > 0) groups[std::make_tuple(h->W, h->T.td, h->T.tda)].push_back(i);
      else rest.push_back(i);
    }
    for (auto &g : groups) {
      double work = 0.0;
      for (size_t i : g.second) work += (double)tg[i].h->S * tg[i].h->K * (double)(tg[i].n_end - tg[i].h->n_now);
      const JitEntry *e = nullptr;
      bool use = g.second.size() >= 2 && (jit_mode > 0 || work >= kJitBatchMinAttempts);
      if (use && (jit_entry(std::get<1>(g.first), std::get<2>(g.first), std::get<0>(g.first), &e) != PCPD_OK ||
                  !e->fn_batch)) {
        g_err.clear();   // no runtime compiler: the generic kernel runs these members
        use = false;
      }
      if (!use) {
        rest.insert(rest.end(), g.second.begin(), g.second.end());
        continue;
      }
      for (size_t c0 = 0; c0 < g.second.size(); c0 += pcpdk::kMaxBatchInst) {
        Chunk ch;
        ch.ids.assign(g.second.begin() + c0,
                      g.second.begin() + std::min(g.second.size(), c0 + (size_t)pcpdk::kMaxBatchInst));
        ch.jit = e;
        chunks.push_back(std::move(ch));
      }
    }
    std::sort(rest.begin(), rest.end());
    for (size_t c0 = 0; c0 < rest.size(); c0 += pcpdk::kMaxBatchInst) {
      Chunk ch;
      ch.ids.assign(rest.begin() + c0, rest.begin() + std::min(rest.size(), c0 + (size_t)pcpdk::kMaxBatchInst));
      chunks.push_back(std::move(ch));
    }
  }
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (const Chunk &ch : chunks) {
    const std::vector<size_t> &ids = ch.ids;
    std::vector<pcpdk::InstDesc> desc(ids.size());
    size_t tile_words = 0;
    uint32_t threads = 64;   // the launch takes the largest CTA any member's plan asks for
    for (size_t q = 0; q < ids.size(); ++q) {
      const size_t i = ids[q];
      pcpd_t *h = tg[i].h;
      fill_desc(h, desc[q], h->n_now, tg[i].n_end, tg[i].rec_first, tg[i].rec_first + tg[i].rec_taken,
                tg[i].slot0);
      tile_words = std::max(tile_words, h->tile_words);
      threads = std::max(threads, h->threads);
    }
    std::vector<std::pair<double, unsigned long long>> ring_items;
    std::vector<unsigned long long> items;
    uint64_t max_ep = 0;
    for (size_t i : ids) max_ep = std::max(max_ep, tg[i].h->ring ? 0 : epochs[i]);
    for (size_t q = 0; q < ids.size(); ++q) {
      const size_t i = ids[q];
      pcpd_t *h = tg[i].h;
      if (!h->ring) continue;
      for (uint64_t e = 0; e < epochs[i]; ++e) {
        const uint64_t len = std::min<uint64_t>(h->tau, tg[i].n_end - h->n_now - e * h->tau);
        for (uint32_t t = 0; t < h->tiles; ++t)
          ring_items.push_back({-(double)h->gpi * h->K * (double)len, pcpdk::pack_item((uint32_t)q, (uint32_t)e, t)});
      }
    }
    // longest first; a later epoch of a tile sorts after all earlier epochs
    std::stable_sort(ring_items.begin(), ring_items.end(),
                     [](const std::pair<double, unsigned long long> &a, const std::pair<double, unsigned long long> &c) {
                       const uint32_t ea = (uint32_t)((a.second >> 24) & 0xFFFFFFu), ec = (uint32_t)((c.second >> 24) & 0xFFFFFFu);
                       if (ea != ec) return ea < ec;
                       return a.first < c.first;
                     });
    const size_t per_round = max_ep ? (ring_items.size() + max_ep - 1) / max_ep : ring_items.size();
    size_t next_ring = 0;
    auto add_ring = [&](size_t count) {
      for (size_t q = 0; q < count && next_ring < ring_items.size(); ++q) items.push_back(ring_items[next_ring++].second);
    };
    for (uint64_t e = 0; e < max_ep; ++e) {
      if (e > 0) add_ring(per_round);
      for (size_t q = 0; q < ids.size(); ++q) {
        const size_t i = ids[q];
        pcpd_t *h = tg[i].h;
        if (h->ring || e >= epochs[i]) continue;
        for (uint32_t t = 0; t < h->tiles; ++t) items.push_back(pcpdk::pack_item((uint32_t)q, (uint32_t)e, t));
      }
    }
    add_ring(ring_items.size());
    if (items.empty()) continue;
    if (items.size() > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "a batch round of %zu work items is too large", items.size());
    if (items.size() > *items_cap) {
      CU(cudaStreamSynchronize(stream));
      cudaFree(*d_items);
      *d_items = nullptr;
      *items_cap = 0;
      const int rc = dev_alloc((void **)d_items, items.size() * sizeof(unsigned long long), "batch work items");
      if (rc) return rc;
      *items_cap = items.size();
    }
    if (items.size() > gc.h_items_cap) {
      CU(cudaStreamSynchronize(stream));
      if (gc.h_items) cudaFreeHost(gc.h_items);
      gc.h_items = nullptr;
      gc.h_items_cap = 0;
      CU(cudaMallocHost(&gc.h_items, items.size() * sizeof(unsigned long long)));
      gc.h_items_cap = items.size();
    }
    if (!gc.h_desc) CU(cudaMallocHost(&gc.h_desc, pcpdk::kMaxBatchInst * sizeof(pcpdk::InstDesc)));
    memcpy(gc.h_items, items.data(), items.size() * sizeof(unsigned long long));
    memcpy(gc.h_desc, desc.data(), desc.size() * sizeof(pcpdk::InstDesc));
    pcpdk::BatchParams B;
    memset(&B, 0, sizeof B);
    B.items = *d_items;
    B.n_items = (uint32_t)items.size();
    B.counter = d_ctl;
    B.err = d_ctl + 1;
    B.tile_words = (uint32_t)tile_words;
    B.spin_limit = kSpinLimit;
    const size_t dyn = 4 * (tile_words + pcpdk::sweep_queue_words(32));
    if (dyn + kStaticSmem > (size_t)optin) return fail(PCPD_EINVAL, "batch tile exceeds shared memory");
    {
      const int rc2 = raise_smem_limit();
      if (rc2) return rc2;
    }
    int per_sm = 0;
    // one window width for the whole round when every instance shares it
    uint32_t wfix = desc.empty() ? 3u : desc[0].W;
    for (const pcpdk::InstDesc &dd : desc)
      if (dd.W != wfix) wfix = 0u;
    const SweepKernel kern = sweep_kernel(true, wfix);
    const JitEntry *jit = ch.jit;
    if (jit && jit->c_inst_bytes < desc.size() * sizeof(pcpdk::InstDesc)) jit = nullptr;   // table too small
    if (jit) {
      if (g_jit_api.occupancy(&per_sm, jit->fn_batch, (int)threads, dyn) != CUDA_SUCCESS) per_sm = 0;
      if (per_sm < 1) jit = nullptr;   // the generic kernel then
    }
    if (!jit) CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
    if (per_sm < 1) return fail(PCPD_EINVAL, "batch plan does not fit one CTA per SM");
    const int grid = (int)std::min<uint64_t>((uint64_t)per_sm * sms, items.size());
    // capture the round, then update the cached executable graph (or instantiate it)
    CU(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(*d_items, gc.h_items, items.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, stream);
    if (jit)   // the runtime-compiled module has its own descriptor table
      cudaMemcpyAsync((void *)jit->c_inst, gc.h_desc, desc.size() * sizeof(pcpdk::InstDesc), cudaMemcpyHostToDevice,
                      stream);
    else
      cudaMemcpyToSymbolAsync(pcpdk::c_inst, gc.h_desc, desc.size() * sizeof(pcpdk::InstDesc), 0,
                              cudaMemcpyHostToDevice, stream);
    cudaMemsetAsync(d_ctl, 0, sizeof(uint32_t), stream);   // work counter
    CUresult launch_rc = CUDA_SUCCESS;
    if (jit) {
      void *args[] = {&B};
      launch_rc = g_jit_api.launch(jit->fn_batch, grid, 1, 1, threads, 1, 1, (unsigned)dyn, (CUstream)stream, args,
                                   nullptr);
    } else {
      kern<<<grid, threads, dyn, stream>>>(B);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(stream, &graph);
    if (ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(PCPD_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
    }
    if (launch_rc != CUDA_SUCCESS) {
      cudaGraphDestroy(graph);
      return fail(PCPD_ECUDA, "launch of the runtime-compiled batch sweep failed (%d)", (int)launch_rc);
    }
    if (jit && jit_launches) ++*jit_launches;
    bool updated = false;
    if (gc.exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(gc.exec, graph, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
      }
    }
    if (!updated) {
      const cudaError_t ei = cudaGraphInstantiate(&gc.exec, graph, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        gc.exec = nullptr;
        return fail(PCPD_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
      }
    }
    cudaGraphDestroy(graph);
    CU(cudaGraphLaunch(gc.exec, stream));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    // the next launch rewrites the constant table and the host vectors go out of scope
    CU(cudaStreamSynchronize(stream));
    uint32_t err = 0;
    CU(cudaMemcpy(&err, d_ctl + 1, 4, cudaMemcpyDeviceToHost));
    if (err) return fail(PCPD_ETIMEOUT, "device wait ran out of its budget (code %u)", err);
  }
  for (size_t i = 0; i < n; ++i) {
    pcpd_t *h = tg[i].h;
    if (epochs[i] & 1u) h->cur = 1 - h->cur;
    h->n_now = tg[i].n_end;
  }
  return PCPD_OK;
}
}  // namespace

extern "C" {

int pcpd_batch_create(void *stream, pcpd_batch_t **out) {
  if (!out) return fail(PCPD_EINVAL, "NULL argument");
  *out = nullptr;
  int rc = device_check();
  if (rc) return rc;
  pcpd_batch_t *b = new pcpd_batch();
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return fail(PCPD_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  cudaError_t e = cudaMalloc(&b->d_ctl, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, 2 * sizeof(uint32_t), b->stream);
  if (e != cudaSuccess) {
    pcpd_batch_destroy(b);
    return fail(PCPD_ENOMEM, "batch control words: %s", cudaGetErrorString(e));
  }
  *out = b;
  return PCPD_OK;
}

void pcpd_batch_destroy(pcpd_batch_t *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (pcpd_t *h : b->inst) pcpd_destroy(h);
  cudaFree(b->d_items);
  cudaFree(b->d_ctl);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

int pcpd_batch_add(pcpd_batch_t *b, const pcpd_params *prm, uint64_t steps_mcs,
                   const uint64_t *record_times_mcs, size_t n_times, size_t *index_out) {
  if (!b || !prm) return fail(PCPD_EINVAL, "NULL argument");
  if (b->ran) return fail(PCPD_ESTATE, "batch already ran");
  if (n_times && !record_times_mcs) return fail(PCPD_EINVAL, "record_times_mcs is NULL");
  for (size_t i = 0; i < n_times; ++i) {
    if (i && record_times_mcs[i] <= record_times_mcs[i - 1]) return fail(PCPD_EINVAL, "record times must increase");
    if (record_times_mcs[i] == 0 || record_times_mcs[i] > steps_mcs)
      return fail(PCPD_EINVAL, "record times must lie in (0, steps_mcs]");
  }
  pcpd_params p2 = *prm;
  p2.stream = b->stream;
  p2.dev_lattice = nullptr;
  p2.dev_bytes = 0;
  p2.jit = -1;   // batched launches run the generic engine (one kernel for many thresholds)
  pcpd_t *h = nullptr;
  int rc = create_handle(&p2, &h, true);
  if (rc) return rc;
  const uint64_t n_end = steps_mcs ? substep_of_time(h->L, steps_mcs, h->W) : 0;
  if (n_end > 0xFFFFFFFFull) {
    pcpd_destroy(h);
    return fail(PCPD_EINVAL, "sub-step count would reach 2^32");
  }
  b->inst.push_back(h);
  b->steps.push_back(steps_mcs);
  b->rec.emplace_back(record_times_mcs, record_times_mcs + n_times);
  if (index_out) *index_out = b->inst.size() - 1;
  return PCPD_OK;
}

int pcpd_batch_run(pcpd_batch_t *b) {
  NvtxRange nvtx("pcpd_batch_run");
  if (!b) return fail(PCPD_EINVAL, "NULL batch");
  if (b->ran) return fail(PCPD_ESTATE, "batch already ran");
  const size_t n = b->inst.size();
  std::vector<MultiTarget> tg(n);
  for (size_t i = 0; i < n; ++i) {
    pcpd_t *h = b->inst[i];
    tg[i].h = h;
    tg[i].n_end = b->steps[i] ? substep_of_time(h->L, b->steps[i], h->W) : 0;
    int rc = ensure_records(h, b->rec[i].size());
    if (rc) return rc;
    if (!b->rec[i].empty()) {
      rc = ensure_rec_sub(h, b->rec[i].size());
      if (rc) return rc;
      std::vector<uint32_t> s32;
      for (uint64_t x : b->rec[i]) s32.push_back((uint32_t)substep_of_time(h->L, x, h->W));
      CU(cudaMemcpyAsync(h->d_rec_sub, s32.data(), s32.size() * 4, cudaMemcpyHostToDevice, b->stream));
      tg[i].rec_sub.assign(s32.begin(), s32.end());
    }
    tg[i].rec_first = 0;
    tg[i].slot0 = 0;
  }
  b->jit_launches = 0;
  int rc = run_multi(b->stream, b->d_ctl, &b->d_items, &b->items_cap, tg, b->gc, b->jit, &b->jit_launches);
  if (rc) return rc;
  for (size_t i = 0; i < n; ++i) {
    pcpd_t *h = b->inst[i];
    h->t_now = b->steps[i];
    for (uint64_t t : b->rec[i]) h->rec_times.push_back(t);
  }
  b->ran = true;
  return PCPD_OK;
}

int pcpd_batch_counts(const pcpd_batch_t *b, size_t i, uint64_t *counts_out, size_t n) {
  if (!b || i >= b->inst.size()) return fail(PCPD_EINVAL, "no instance %zu", i);
  if (!b->ran) return fail(PCPD_ESTATE, "batch has not run");
  return pcpd_density(b->inst[i], nullptr, counts_out, n);
}

int pcpd_batch_pair_counts(const pcpd_batch_t *b, size_t i, uint64_t *counts_out, size_t n) {
  if (!b || i >= b->inst.size()) return fail(PCPD_EINVAL, "no instance %zu", i);
  if (!b->ran) return fail(PCPD_ESTATE, "batch has not run");
  return pcpd_pair_counts(b->inst[i], counts_out, n);
}

int pcpd_batch_lattice(const pcpd_batch_t *b, size_t i, uint32_t *host_out) {
  if (!b || i >= b->inst.size()) return fail(PCPD_EINVAL, "no instance %zu", i);
  return pcpd_get_lattice(b->inst[i], host_out);
}

size_t pcpd_batch_size(const pcpd_batch_t *b) { return b ? b->inst.size() : 0; }

int pcpd_batch_set_jit(pcpd_batch_t *b, int mode) {
  if (!b) return fail(PCPD_EINVAL, "NULL batch");
  b->jit = mode > 0 ? 1 : (mode < 0 ? -1 : 0);
  return PCPD_OK;
}

size_t pcpd_batch_jit_launches(const pcpd_batch_t *b) { return b ? b->jit_launches : 0; }

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Serving: continuous batching of simulation requests.  A host thread owns the GPU work: it
// admits queued requests while active slots and the device-memory budget allow, advances
// every active request by a bounded chunk per round in one engine launch (their work
// overlaps on the device), keeps each request's lattice and clock on the device between
// rounds, and retires finished requests, freeing their slot and memory for the queue.
// ------------------------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  pcpd_params prm{};
  uint64_t steps = 0;
  std::vector<uint64_t> rec_times;
  bool keep_lattice = false;
  Clock::time_point t_submit, t_admit, t_done;
  int state = 0;  // 0 queued, 1 active, 2 done, 3 failed
  std::string err;
  pcpd_t *h = nullptr;
  uint64_t n_end = 0;
  std::vector<uint64_t> rec_sub;
  size_t rec_first = 0;
  size_t bytes = 0;
  std::vector<uint64_t> counts;
  std::vector<uint32_t> lattice;
  bool cancel = false;   // set by pcpd_server_cancel while the request is on the GPU
};

size_t request_bytes(const pcpd_params &p, size_t n_rec) {
  const size_t G = p.samples / 32u, pitch = (p.L + 3u) & ~3u;
  return 2 * G * pitch * 4 + n_rec * 8 + (p.per_sample ? n_rec * (size_t)p.samples * 4 : 0) + 4096;
}

}  // namespace

struct pcpd_server {
  pcpd_server_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t *d_ctl = nullptr;
  unsigned long long *d_items = nullptr;
  size_t items_cap = 0;
  GraphCache gc;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<Request *> pending;
  std::vector<Request *> active;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_id = 1;
  size_t mem_used = 0;
  int device = 0;
  pcpd_server_stats st{};
  std::string fatal;
};

namespace {

void server_retire(pcpd_server_t *sv, Request *r, int ok, const std::string &msg) {
  if (ok) {
    r->counts.resize(r->rec_times.size());
    if (!r->counts.empty() && pcpd_density(r->h, nullptr, r->counts.data(), r->counts.size()) != PCPD_OK) {
      ok = 0;
      r->err = g_err;
    }
    if (ok && r->keep_lattice) {
      r->lattice.resize((size_t)(r->prm.samples / 32u) * r->prm.L);
      if (pcpd_get_lattice(r->h, r->lattice.data()) != PCPD_OK) {
        ok = 0;
        r->err = g_err;
      }
    }
  } else {
    r->err = msg;
  }
  pcpd_destroy(r->h);
  r->h = nullptr;
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->mem_used -= r->bytes;
  r->t_done = Clock::now();
  r->state = ok ? 2 : 3;
  if (ok) sv->st.completed++;
  else sv->st.failed++;
  sv->cv_done.notify_all();
}

void server_loop(pcpd_server_t *sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Request *> admit;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv.wait(lock, [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
      if (sv->stop) break;
      // admission: FIFO while a slot and the memory budget are free (an oversized request is
      // admitted alone so that it cannot block the queue forever)
      while (!sv->pending.empty() && sv->active.size() + admit.size() < sv->cfg.max_active) {
        Request *r = sv->pending.front();
        if (sv->mem_used + r->bytes > sv->cfg.hbm_budget_bytes && !(sv->active.empty() && admit.empty())) break;
        sv->pending.pop_front();
        sv->mem_used += r->bytes;
        admit.push_back(r);
      }
    }
    for (Request *r : admit) {
      pcpd_params p2 = r->prm;
      p2.stream = sv->stream;
      p2.dev_lattice = nullptr;
      p2.jit = -1;   // serving rounds run the generic engine
      int rc = create_handle(&p2, &r->h, true);
      if (rc == PCPD_OK) rc = ensure_records(r->h, r->rec_times.size());
      if (rc == PCPD_OK && !r->rec_times.empty()) {
        rc = ensure_rec_sub(r->h, r->rec_times.size());
        std::vector<uint32_t> s32;
        for (uint64_t t : r->rec_times) {
          r->rec_sub.push_back(substep_of_time(r->h->L, t, r->h->W));
          s32.push_back((uint32_t)r->rec_sub.back());
        }
        if (rc == PCPD_OK &&
            cudaMemcpyAsync(r->h->d_rec_sub, s32.data(), s32.size() * 4, cudaMemcpyHostToDevice, sv->stream) != cudaSuccess)
          rc = PCPD_ECUDA;
        if (rc == PCPD_OK && cudaStreamSynchronize(sv->stream) != cudaSuccess) rc = PCPD_ECUDA;
      }
      r->t_admit = Clock::now();
      if (rc != PCPD_OK) {
        server_retire(sv, r, 0, g_err);
        continue;
      }
      r->n_end = r->steps ? substep_of_time(r->h->L, r->steps, r->h->W) : 0;
      std::lock_guard<std::mutex> lock(sv->mu);
      r->state = 1;
      sv->active.push_back(r);
    }
    std::vector<Request *> act;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      act = sv->active;
    }
    if (act.empty()) continue;
    // one round: every active request advances by at most chunk_attempts attempts
    std::vector<MultiTarget> tg(act.size());
    unsigned long long round_attempts = 0;
    for (size_t i = 0; i < act.size(); ++i) {
      Request *r = act[i];
      pcpd_t *h = r->h;
      const unsigned long long per_sub = (unsigned long long)h->S * h->K;
      uint64_t chunk = sv->cfg.chunk_attempts / (per_sub ? per_sub : 1);
      if (chunk < 1) chunk = 1;
      tg[i].h = h;
      tg[i].n_end = std::min<uint64_t>(r->n_end, h->n_now + chunk);
      tg[i].rec_sub = r->rec_sub;
      tg[i].rec_first = r->rec_first;
      tg[i].slot0 = r->rec_first;
      round_attempts += per_sub * (tg[i].n_end - h->n_now);
    }
    const Clock::time_point t0 = Clock::now();
    int rc;
    {
      NvtxRange nvtx("pcpd_server_round");
      rc = run_multi(sv->stream, sv->d_ctl, &sv->d_items, &sv->items_cap, tg, sv->gc);
    }
    const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->st.rounds++;
      sv->st.busy_seconds += dt;
      if (rc == PCPD_OK) sv->st.attempts += round_attempts;
    }
    for (size_t i = 0; i < act.size(); ++i) {
      Request *r = act[i];
      if (rc != PCPD_OK) {
        {
          std::lock_guard<std::mutex> lock(sv->mu);
          sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
        }
        server_retire(sv, r, 0, g_err);
        continue;
      }
      r->rec_first += tg[i].rec_taken;
      bool cancelled;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        cancelled = r->cancel;
        if (cancelled) sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
      }
      if (cancelled) {   // between rounds: nothing of this request is in flight
        server_retire(sv, r, 0, "cancelled");
        continue;
      }
      if (r->h->n_now >= r->n_end) {
        r->h->t_now = r->steps;
        r->h->rec_times = r->rec_times;
        {
          std::lock_guard<std::mutex> lock(sv->mu);
          sv->active.erase(std::find(sv->active.begin(), sv->active.end(), r));
        }
        server_retire(sv, r, 1, "");
      }
    }
  }
  // stopped: abandon what is left
  std::vector<Request *> left;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    left = sv->active;
    sv->active.clear();
    for (Request *r : sv->pending) left.push_back(r);
    sv->pending.clear();
  }
  for (Request *r : left) server_retire(sv, r, 0, "server stopped");
}

}  // namespace

extern "C" {

int pcpd_server_start(const pcpd_server_config *cfg, pcpd_server_t **out) {
  if (!cfg || !out) return fail(PCPD_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_active == 0 || cfg->max_active > (uint32_t)pcpdk::kMaxBatchInst)
    return fail(PCPD_EINVAL, "max_active must be in [1, %d]", pcpdk::kMaxBatchInst);
  if (cfg->hbm_budget_bytes == 0 || cfg->chunk_attempts == 0) return fail(PCPD_EINVAL, "budget and chunk must be positive");
  int rc = device_check();
  if (rc) return rc;
  pcpd_server_t *sv = new pcpd_server();
  sv->cfg = *cfg;
  CU(cudaGetDevice(&sv->device));
  cudaError_t e = cudaSuccess;
  if (cfg->stream) {
    sv->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    sv->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&sv->d_ctl, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(sv->d_ctl, 0, 2 * sizeof(uint32_t), sv->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
  if (e != cudaSuccess) {
    if (sv->own_stream) cudaStreamDestroy(sv->stream);
    cudaFree(sv->d_ctl);
    delete sv;
    return fail(PCPD_ECUDA, "server start: %s", cudaGetErrorString(e));
  }
  sv->th = std::thread(server_loop, sv);
  *out = sv;
  return PCPD_OK;
}

int pcpd_server_submit(pcpd_server_t *sv, const pcpd_params *prm, uint64_t steps_mcs,
                       const uint64_t *record_times_mcs, size_t n_times, int keep_lattice, uint64_t *id_out) {
  if (!sv || !prm || !id_out) return fail(PCPD_EINVAL, "NULL argument");
  if (n_times && !record_times_mcs) return fail(PCPD_EINVAL, "record_times_mcs is NULL");
  if (prm->L < 3 || prm->L >= (1u << 30) || prm->samples == 0 || prm->samples % 32 || prm->samples > (1u << 22))
    return fail(PCPD_EINVAL, "bad L or samples");
  if (prm->tuple == 1u || prm->tuple > 4u || prm->L < (prm->tuple ? prm->tuple : 2u) + 1u)
    return fail(PCPD_EINVAL, "bad tuple size or L shorter than one window");
  uint64_t td, tda;
  int rc = thresholds(prm->p, prm->d, &td, &tda);
  if (rc) return rc;
  for (size_t i = 0; i < n_times; ++i) {
    if (i && record_times_mcs[i] <= record_times_mcs[i - 1]) return fail(PCPD_EINVAL, "record times must increase");
    if (record_times_mcs[i] == 0 || record_times_mcs[i] > steps_mcs)
      return fail(PCPD_EINVAL, "record times must lie in (0, steps_mcs]");
  }
  if (steps_mcs && substep_of_time(prm->L, steps_mcs, (prm->tuple ? prm->tuple : 2u) + 1u) > 0xFFFFFFFFull)
    return fail(PCPD_EINVAL, "too many sub-steps");
  std::unique_ptr<Request> r(new Request());
  r->prm = *prm;
  r->steps = steps_mcs;
  r->rec_times.assign(record_times_mcs, record_times_mcs + n_times);
  r->keep_lattice = keep_lattice != 0;
  r->bytes = request_bytes(*prm, n_times);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return fail(PCPD_ESTATE, "server stopped");
  r->id = sv->next_id++;
  *id_out = r->id;
  sv->pending.push_back(r.get());
  sv->all[r->id] = std::move(r);
  sv->st.submitted++;
  sv->cv.notify_all();
  return PCPD_OK;
}

int pcpd_server_cancel(pcpd_server_t *sv, uint64_t id) {
  if (!sv) return fail(PCPD_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return fail(PCPD_EINVAL, "unknown request %llu", (unsigned long long)id);
  Request *r = it->second.get();
  if (r->state == 0) {   // still queued: it holds no device memory
    sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
    r->state = 3;
    r->err = "cancelled";
    r->t_done = Clock::now();
    sv->st.failed++;
    sv->cv_done.notify_all();
    return PCPD_OK;
  }
  if (r->state == 1) {   // retired by the server thread after the current round
    r->cancel = true;
    return PCPD_OK;
  }
  return fail(PCPD_ESTATE, "request %llu has already finished", (unsigned long long)id);
}

int pcpd_server_poll(pcpd_server_t *sv, uint64_t id, int *state_out) {
  if (!sv || !state_out) return fail(PCPD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return fail(PCPD_EINVAL, "unknown request %llu", (unsigned long long)id);
  *state_out = it->second->state;
  return PCPD_OK;
}

int pcpd_server_result(pcpd_server_t *sv, uint64_t id, uint64_t *counts_out, size_t n, uint32_t *lattice_out,
                       double *latency_s, double *queue_s) {
  if (!sv) return fail(PCPD_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return fail(PCPD_EINVAL, "unknown request %llu", (unsigned long long)id);
  Request *r = it->second.get();
  sv->cv_done.wait(lock, [&] { return r->state >= 2; });
  if (r->state == 3) return fail(PCPD_ESTATE, "request %llu failed: %s", (unsigned long long)id, r->err.c_str());
  if (n > r->counts.size()) return fail(PCPD_EINVAL, "request has %zu records", r->counts.size());
  if (counts_out) std::copy(r->counts.begin(), r->counts.begin() + n, counts_out);
  if (lattice_out) {
    if (!r->keep_lattice) return fail(PCPD_ESTATE, "lattice was not kept (keep_lattice = 0)");
    std::copy(r->lattice.begin(), r->lattice.end(), lattice_out);
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (queue_s) *queue_s = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
  return PCPD_OK;
}

int pcpd_server_wait_idle(pcpd_server_t *sv) {
  if (!sv) return fail(PCPD_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lock(sv->mu);
  sv->cv_done.wait(lock, [&] { return sv->st.completed + sv->st.failed == sv->st.submitted; });
  return PCPD_OK;
}

int pcpd_server_get_stats(pcpd_server_t *sv, pcpd_server_stats *out) {
  if (!sv || !out) return fail(PCPD_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  *out = sv->st;
  out->active = sv->active.size();
  out->queued = sv->pending.size();
  out->mem_used_bytes = sv->mem_used;
  return PCPD_OK;
}

void pcpd_server_stop(pcpd_server_t *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  cudaStreamSynchronize(sv->stream);
  cudaFree(sv->d_items);
  cudaFree(sv->d_ctl);
  if (sv->own_stream) cudaStreamDestroy(sv->stream);
  delete sv;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Test entry for the engine's failure path: one item of epoch 1 whose epoch-0 predecessor is
// never scheduled, so its bounded wait must run out, record kErrDepTimeout and end the CTA.
// ------------------------------------------------------------------------------------------
extern "C" int pcpd_dev_timeout_test(unsigned long long spin_limit_cycles) {
  int rc = device_check();
  if (rc) return rc;
  if (spin_limit_cycles == 0 || spin_limit_cycles > (1ull << 34)) return fail(PCPD_EINVAL, "spin limit out of range");
  pcpd_params prm;
  memset(&prm, 0, sizeof prm);
  prm.L = 96;
  prm.samples = 32;
  prm.p = 0.1;
  prm.d = 0.5;
  prm.seed = 1;
  prm.plan_tau = 8;
  pcpd_t *h = nullptr;
  rc = pcpd_create_ex(&prm, &h);
  if (rc) return rc;
  pcpd_batch_t *b = nullptr;
  rc = pcpd_batch_create(h->stream, &b);
  if (rc) {
    pcpd_destroy(h);
    return rc;
  }
  int out = PCPD_OK;
  {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    pcpdk::InstDesc D;
    fill_desc(h, D, 0, 16, 0, 0, 0);
    const unsigned long long item = pcpdk::pack_item(0, 1, 0);   // epoch 1 of tile 0 only
    cudaError_t e = cudaMemsetAsync(h->d_done, 0, (h->tiles + 2) * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof item);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_items, &item, sizeof item, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyToSymbolAsync(pcpdk::c_inst, &D, sizeof D, 0, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, 2 * sizeof(uint32_t), h->stream);
    if (e == cudaSuccess) e = (cudaError_t)raise_smem_limit() == 0 ? cudaSuccess : cudaErrorInvalidValue;
    if (e == cudaSuccess) {
      pcpdk::BatchParams B;
      memset(&B, 0, sizeof B);
      B.items = b->d_items;
      B.n_items = 1;
      B.counter = b->d_ctl;
      B.err = b->d_ctl + 1;
      B.tile_words = (uint32_t)h->tile_words;
      B.spin_limit = spin_limit_cycles;
      sweep_kernel(true, 3u)<<<1, 256, 4 * (h->tile_words + pcpdk::sweep_queue_words(8)), h->stream>>>(B);
      e = cudaGetLastError();
    }
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, b->d_ctl + 1, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) out = fail(PCPD_ECUDA, "timeout test: %s", cudaGetErrorString(e));
    else if (err == pcpdk::kErrDepTimeout) out = fail(PCPD_ETIMEOUT, "dependency wait gave up after its budget, as designed");
    else out = fail(PCPD_ESTATE, "timeout test: error word %u, expected %u", err, pcpdk::kErrDepTimeout);
  }
  pcpd_batch_destroy(b);
  pcpd_destroy(h);
  return out;
}

// ------------------------------------------------------------------------------------------
// Autotuner: time candidate plans on the real instance and keep the fastest.
// ------------------------------------------------------------------------------------------
namespace {

struct TunedPlan {
  uint32_t threads, seg, tau;
  double rate;
};
std::mutex g_tune_mu;
// key: (L | (W - 3) << 30, samples) -- L < 2^30, W the window width
std::map<std::pair<uint32_t, uint32_t>, TunedPlan> g_tune;

uint32_t tune_key_L(const pcpd_params *prm) {
  const uint32_t W = (prm->tuple ? prm->tuple : 2u) + 1u;
  return prm->L | ((W - 3u) << 30);
}
bool g_tune_file_read = false;

void tune_file_load() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char *path = getenv("PCPD_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  unsigned L, S, th, seg, tau;
  double rate;
  while (fscanf(f, "%u %u %u %u %u %lf", &L, &S, &th, &seg, &tau, &rate) == 6) g_tune[{L, S}] = {th, seg, tau, rate};
  fclose(f);
}

void tune_file_append(uint32_t L, uint32_t S, const TunedPlan &t) {
  const char *path = getenv("PCPD_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%u %u %u %u %u %.6e\n", L, S, t.threads, t.seg, t.tau, t.rate);
  fclose(f);
}

// Rate of one plan: attempted updates/s over trial sub-steps after one warm-up epoch.
int time_plan(const pcpd_params *prm, uint32_t trial, double *rate) {
  pcpd_params p2 = *prm;
  p2.autotune = 0;
  p2.per_sample = 0;
  p2.stream = nullptr;
  p2.dev_lattice = nullptr;
  pcpd_t *h = nullptr;
  int rc = pcpd_create_ex(&p2, &h);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = pcpd_run_substeps(h, std::min<uint64_t>(trial, h->tau));
  if (rc == PCPD_OK) rc = pcpd_sync(h);
  if (rc == PCPD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(PCPD_ECUDA, "event create");
  float ms = 0.f;
  if (rc == PCPD_OK) {
    cudaEventRecord(e0, h->stream);
    rc = pcpd_run_substeps(h, trial);
    cudaEventRecord(e1, h->stream);
    if (rc == PCPD_OK) rc = pcpd_sync(h);
    if (rc == PCPD_OK) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == PCPD_OK) *rate = ms > 0.f ? (double)h->S * h->K * trial / (ms * 1e-3) : 0.0;
  pcpd_destroy(h);
  return rc;
}

int tuned_plan(const pcpd_params *prm, pcpd_params *out) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_file_load();
    auto it = g_tune.find({tune_key_L(prm), prm->samples});
    if (it != g_tune.end()) {
      *out = *prm;
      out->autotune = 0;
      out->plan_threads = it->second.threads;
      out->plan_seg_sites = it->second.seg;
      out->plan_tau = it->second.tau;
      return PCPD_OK;
    }
  }
  return pcpd_autotune(prm, 0, out, nullptr);
}

}  // namespace

extern "C" int pcpd_autotune(const pcpd_params *prm, uint32_t trial_substeps, pcpd_params *best, double *best_rate) {
  if (!prm || !best) return fail(PCPD_EINVAL, "NULL argument");
  int rc = device_check();
  if (rc) return rc;
  // the default plan tells RING from SEGMENT and gives the largest tile
  pcpd base;
  base.L = prm->L;
  base.W = (prm->tuple ? prm->tuple : 2u) + 1u;
  base.K = prm->L / base.W;
  base.S = prm->samples;
  base.G = prm->samples / 32u;
  if (prm->samples == 0 || prm->samples % 32 || prm->L < 3) return fail(PCPD_EINVAL, "bad L or samples");
  rc = make_plan(&base, nullptr);
  if (rc) return rc;
  pcpd paired = base;   // the tile two CTAs per SM can hold
  rc = make_plan(&paired, nullptr, kPlanPaired);
  if (rc) return rc;
  struct Cand {
    uint32_t threads, seg, tau;
  };
  std::vector<Cand> cands;
  if (base.ring) {
    for (uint32_t th : {128u, 256u, 512u})
      if (th <= pcpdk::kSweepThreads && (th <= base.threads * 2u || th == 128u)) cands.push_back({th, 0u, 0u});
    if (!paired.ring)   // too few columns for the SMs: the segment plan of a lone instance
      for (uint32_t tau : {64u, 128u}) cands.push_back({paired.threads, paired.core, tau});
  } else {
    const uint32_t half = ((base.core / 2u) + 3u) & ~3u;
    std::vector<uint32_t> segs = {base.core, half};
    if (paired.core != base.core && paired.core != half) segs.push_back(paired.core);
    for (uint32_t th : {256u, 512u})
      for (uint32_t tau : {64u, 128u, 256u})
        for (uint32_t seg : segs) {
          if (seg + 2u * ((base.W - 1u) * tau + base.W + 1u) + 4u * base.W > prm->L || (prm->L + seg - 1) / seg < 2)
            continue;
          cands.push_back({th, seg, tau});
        }
  }
  if (trial_substeps == 0) trial_substeps = base.ring ? 256u : 512u;
  double best_r = -1.0;
  Cand win{0, 0, 0};
  for (const Cand &c : cands) {
    pcpd_params p2 = *prm;
    p2.plan_threads = c.threads;
    p2.plan_seg_sites = c.seg;
    p2.plan_tau = c.tau;
    double r = 0.0;
    if (time_plan(&p2, trial_substeps, &r) != PCPD_OK) continue;   // a plan that does not fit is skipped
    if (r > best_r) {
      best_r = r;
      win = c;
    }
  }
  if (best_r < 0.0) return fail(PCPD_EINVAL, "no candidate plan could run");
  *best = *prm;
  best->autotune = 0;
  best->plan_threads = win.threads;
  best->plan_seg_sites = win.seg;
  best->plan_tau = win.tau;
  if (best_rate) *best_rate = best_r;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const TunedPlan t{win.threads, win.seg, win.tau, best_r};
  g_tune[{tune_key_L(prm), prm->samples}] = t;
  tune_file_append(tune_key_L(prm), prm->samples, t);
  return PCPD_OK;
}

// ------------------------------------------------------------------------------------------
// The paper's own GPU scheme (Sec. 3-4, Alg. 2) as a variant: one system per group of S_w
// threads, a shared random local site per step, correlated annihilation draws.
struct pcpd_paper {
  uint32_t n_loc = 0, S_w = 0, systems = 0, L = 0, words = 0;
  uint32_t m = 0, n_dec = 0, t_d = 0, d_full = 0, tc = 0, tc_full = 0;
  pcpdk::RoundKeys rk{};
  uint64_t step = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t *d_lat = nullptr;
  std::vector<uint64_t> rec_steps;
  unsigned long long *d_rec_total = nullptr, *d_rec_step = nullptr;
  uint32_t *d_rec_sys = nullptr;
  size_t rec_cap = 0;
  uint32_t spc = 1, threads = 0, grid = 0;
  size_t smem = 0;
  void (*kernel)(const pcpdk::PaperParams) = nullptr;
};

namespace {

using PaperKernel = void (*)(const pcpdk::PaperParams);

// Compile-time plane/decorrelation counts for the common cases and CTAs of up to 256
// threads; a kernel that reads them at run time otherwise.
template <int M>
PaperKernel paper_kernel_m(uint32_t nd) {
  switch (nd) {
    case 0: return pcpdk::k_paper_sweep<M, 0, 256, false>;
    case 1: return pcpdk::k_paper_sweep<M, 1, 256, false>;
    case 2: return pcpdk::k_paper_sweep<M, 2, 256, false>;
    case 3: return pcpdk::k_paper_sweep<M, 3, 256, false>;
    default: return pcpdk::k_paper_sweep<-1, 0, 256, false>;
  }
}

PaperKernel paper_kernel(uint32_t m, uint32_t nd, uint32_t threads, uint32_t S_w, uint32_t spc, int generic) {
  // the small-CTA kernels hold one system per CTA unless a system is one warp; several
  // multi-warp systems per CTA need named barriers
  if (S_w > 32 && spc > 1) return pcpdk::k_paper_sweep<-1, 0, 1024, true>;   // per-system barriers
  if (threads > 256) return pcpdk::k_paper_sweep<-1, 0, 1024, false>;
  if (generic) return pcpdk::k_paper_sweep<-1, 0, 256, false>;
  switch (m) {
    case 0: return paper_kernel_m<0>(nd);
    case 1: return paper_kernel_m<1>(nd);
    case 2: return paper_kernel_m<2>(nd);
    case 3: return paper_kernel_m<3>(nd);
    default: return pcpdk::k_paper_sweep<-1, 0, 256, false>;
  }
}

// Raise a kernel's dynamic shared-memory limit once per process (the attribute is global).
int paper_smem_optin(PaperKernel k, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void *, size_t>> done;
  std::lock_guard<std::mutex> lk(mu);
  for (auto &e : done)
    if (e.first == (const void *)k && e.second >= bytes) return PCPD_OK;
  int optin = 0;
  int rc = smem_optin(&optin);
  if (rc) return rc;
  CU(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  // all of the SM's unified L1/shared storage as shared memory: the systems are the working set
  CU(cudaFuncSetAttribute((const void *)k, cudaFuncAttributePreferredSharedMemoryCarveout,
                          (int)cudaSharedmemCarveoutMaxShared));
  done.emplace_back((const void *)k, (size_t)optin);
  return PCPD_OK;
}

int paper_ensure_records(pcpd_paper_t *h, size_t need) {
  if (need <= h->rec_cap) return PCPD_OK;
  size_t cap = h->rec_cap ? h->rec_cap : 64;
  while (cap < need) cap *= 2;
  unsigned long long *nt = nullptr, *ns = nullptr;
  uint32_t *nsys = nullptr;
  FreeUnlessKept pending{{(void **)&nt, (void **)&ns, (void **)&nsys}};
  int rc = dev_alloc((void **)&nt, cap * sizeof(unsigned long long), "record totals");
  if (!rc) rc = dev_alloc((void **)&ns, cap * sizeof(unsigned long long), "record steps");
  if (!rc) rc = dev_alloc((void **)&nsys, cap * (size_t)h->systems * sizeof(uint32_t), "per-system records");
  if (rc) return rc;
  CU(cudaMemsetAsync(nt, 0, cap * sizeof(unsigned long long), h->stream));
  CU(cudaMemsetAsync(nsys, 0, cap * (size_t)h->systems * sizeof(uint32_t), h->stream));
  const size_t have = h->rec_steps.size();
  if (have) {
    CU(cudaMemcpyAsync(nt, h->d_rec_total, have * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream));
    CU(cudaMemcpyAsync(nsys, h->d_rec_sys, have * (size_t)h->systems * sizeof(uint32_t),
                       cudaMemcpyDeviceToDevice, h->stream));
  }
  CU(cudaStreamSynchronize(h->stream));
  pending.keep = true;
  cudaFree(h->d_rec_total);
  cudaFree(h->d_rec_step);
  cudaFree(h->d_rec_sys);
  h->d_rec_total = nt;
  h->d_rec_step = ns;
  h->d_rec_sys = nsys;
  h->rec_cap = cap;
  return PCPD_OK;
}

}  // namespace

int pcpd_paper_thresholds(double p, double d, uint32_t m, uint32_t n_dec, uint32_t *t_d,
                          uint64_t *t_c) {
  if (!t_d || !t_c) return fail(PCPD_EINVAL, "NULL output");
  if (m > 16 || n_dec > 16) return fail(PCPD_EINVAL, "m and n_dec must be at most 16 (m=%u, n_dec=%u)", m, n_dec);
  const double td = d * (double)(1u << m);
  if (!(td >= 0.0 && td <= (double)(1u << m)) || td != std::floor(td))
    return fail(PCPD_EINVAL, "d=%g is not a multiple of 2^-%u in [0, 1]", d, m);
  const double c = p * (double)(1u << n_dec);
  if (!(c >= 0.0 && c <= 1.0)) return fail(PCPD_EINVAL, "need 0 <= p * 2^n_dec <= 1 (p=%g, n_dec=%u)", p, n_dec);
  *t_d = (uint32_t)td;
  *t_c = floor_scaled(c * 4294967296.0);
  return PCPD_OK;
}

int pcpd_paper_create(const pcpd_paper_params *prm, pcpd_paper_t **out) {
  if (!prm || !out) return fail(PCPD_EINVAL, "NULL argument");
  *out = nullptr;
  if (prm->n_loc < 4) return fail(PCPD_EINVAL, "n_loc must be at least 4 (n_loc=%u)", prm->n_loc);
  if (prm->S_w < 32 || prm->S_w > 1024 || prm->S_w % 32)
    return fail(PCPD_EINVAL, "S_w must be a multiple of 32 in [32, 1024] (S_w=%u)", prm->S_w);
  if (prm->systems == 0 || prm->systems > (1u << 24))
    return fail(PCPD_EINVAL, "systems must lie in [1, 2^24] (systems=%u)", prm->systems);
  if (prm->init != PCPD_INIT_FULL && prm->init != PCPD_INIT_EMPTY)
    return fail(PCPD_EINVAL, "init must be PCPD_INIT_FULL or PCPD_INIT_EMPTY (init=%d)", prm->init);
  uint32_t t_d = 0;
  uint64_t t_c = 0;
  int rc = pcpd_paper_thresholds(prm->p, prm->d, prm->m, prm->n_dec, &t_d, &t_c);
  if (rc) return rc;
  rc = device_check();
  if (rc) return rc;
  int optin = 0;
  rc = smem_optin(&optin);
  if (rc) return rc;
  const uint64_t words = (uint64_t)prm->n_loc * prm->S_w;
  if (words * 4 > (uint64_t)optin)
    return fail(PCPD_EINVAL, "a system of n_loc*S_w = %llu words does not fit one CTA's shared memory (%d bytes)",
                (unsigned long long)words, optin);
  uint32_t spc = prm->plan_spc;
  if (spc == 0) {
    spc = prm->S_w > 32 ? 1u : 8u;   // systems of several warps: one per CTA (CTA barrier)
    while (spc > 1 && spc * words * 4 > (uint64_t)optin) --spc;
  }
  if (spc > 15 || spc * prm->S_w > 1024 || spc * words * 4 > (uint64_t)optin)
    return fail(PCPD_EINVAL, "plan_spc=%u systems per CTA does not fit (at most 15, 1024 threads, %d bytes)", spc, optin);

  pcpd_paper_t *h = new pcpd_paper();
  auto bail = [&](int code) {
    pcpd_paper_destroy(h);
    return code;
  };
  h->n_loc = prm->n_loc;
  h->S_w = prm->S_w;
  h->systems = prm->systems;
  h->words = (uint32_t)words;
  h->L = 32u * h->words;
  h->m = prm->m;
  h->n_dec = prm->n_dec;
  h->t_d = t_d;
  h->d_full = t_d == (1u << prm->m) ? 1u : 0u;
  h->tc = (uint32_t)(t_c & 0xFFFFFFFFull);
  h->tc_full = t_c >= kTwo32 ? 1u : 0u;
  h->rk = pcpdk::make_round_keys((uint32_t)(prm->seed & 0xFFFFFFFFu), (uint32_t)(prm->seed >> 32));
  h->spc = spc;
  h->threads = spc * h->S_w;
  h->grid = (h->systems + spc - 1) / spc;
  h->smem = (size_t)spc * words * 4;
  h->kernel = paper_kernel(h->m, h->n_dec, h->threads, h->S_w, h->spc, prm->generic);
  rc = paper_smem_optin(h->kernel, h->smem);
  if (rc) return bail(rc);
  if (prm->stream) {
    h->stream = (cudaStream_t)prm->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(PCPD_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)));
    h->own_stream = true;
  }
  const size_t bytes = (size_t)h->systems * words * 4;
  const int ra = dev_alloc((void **)&h->d_lat, bytes, "systems");
  if (ra) return bail(ra);
  cudaError_t e = cudaMemsetAsync(h->d_lat, prm->init == PCPD_INIT_FULL ? 0xFF : 0x00, bytes, h->stream);
  if (e != cudaSuccess) return bail(fail(PCPD_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)));
  *out = h;
  return PCPD_OK;
}

void pcpd_paper_destroy(pcpd_paper_t *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->d_lat);
  cudaFree(h->d_rec_total);
  cudaFree(h->d_rec_step);
  cudaFree(h->d_rec_sys);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

int pcpd_paper_run(pcpd_paper_t *h, uint64_t n_steps, const uint64_t *record_steps, size_t n_rec) {
  NvtxRange nvtx("pcpd_paper_run");
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  if (n_rec && !record_steps) return fail(PCPD_EINVAL, "record_steps is NULL");
  const uint64_t end = h->step + n_steps;
  if (end > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "step count %llu would exceed 2^32 - 1", (unsigned long long)end);
  for (size_t i = 0; i < n_rec; ++i) {
    const uint64_t s = record_steps[i];
    if (i && s <= record_steps[i - 1]) return fail(PCPD_EINVAL, "record steps must be strictly increasing");
    if (s > end || s < h->step || (s == h->step && i != 0))
      return fail(PCPD_EINVAL, "record step %llu outside [%llu, %llu] (the current step only as the first)",
                  (unsigned long long)s, (unsigned long long)h->step, (unsigned long long)end);
  }
  const size_t slot0 = h->rec_steps.size();
  int rc = paper_ensure_records(h, slot0 + n_rec);
  if (rc) return rc;
  if (n_rec) {
    CU(cudaMemcpyAsync(h->d_rec_step + slot0, record_steps, n_rec * sizeof(uint64_t), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));  // record_steps belongs to the caller
  }
  // launches of at most 2^20 steps; a launch records the steps in [a, b), the last one also b
  constexpr uint64_t kChunk = 1ull << 20;
  size_t r = 0;
  uint64_t a = h->step;
  do {
    const uint64_t b = std::min(end, a + kChunk);
    size_t r1 = r;
    while (r1 < n_rec && (record_steps[r1] < b || (b == end && record_steps[r1] == b))) ++r1;
    pcpdk::PaperParams P{};
    P.lat = h->d_lat;
    P.rec_step = h->d_rec_step + slot0 + r;
    P.rec_total = h->d_rec_total + slot0 + r;
    P.rec_sys = h->d_rec_sys + (slot0 + r) * (size_t)h->systems;
    P.rk = h->rk;
    P.n_loc = h->n_loc;
    P.S_w = h->S_w;
    P.systems = h->systems;
    P.spc = h->spc;
    P.m = h->m;
    P.t_d = h->t_d;
    P.d_full = h->d_full;
    P.n_dec = h->n_dec;
    P.tc = h->tc;
    P.tc_full = h->tc_full;
    P.step_begin = (uint32_t)a;
    P.step_end = (uint32_t)b;
    P.n_rec = (uint32_t)(r1 - r);
    P.systems_total = h->systems;
    h->kernel<<<h->grid, h->threads, h->smem, h->stream>>>(P);
    CU(cudaGetLastError());
    g_launches.fetch_add(1, std::memory_order_relaxed);
    r = r1;
    a = b;
  } while (a < end);
  h->rec_steps.insert(h->rec_steps.end(), record_steps, record_steps + n_rec);
  h->step = end;
  return PCPD_OK;
}

size_t pcpd_paper_num_records(const pcpd_paper_t *h) { return h ? h->rec_steps.size() : 0; }

uint64_t pcpd_paper_step(const pcpd_paper_t *h) { return h ? h->step : 0; }

int pcpd_paper_counts(const pcpd_paper_t *h, uint64_t *counts_out, uint32_t *per_system_out, size_t n) {
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  if (n > h->rec_steps.size()) return fail(PCPD_EINVAL, "only %zu records taken", h->rec_steps.size());
  if (n == 0) return PCPD_OK;
  if (counts_out)
    CU(cudaMemcpyAsync(counts_out, h->d_rec_total, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
  if (per_system_out)
    CU(cudaMemcpyAsync(per_system_out, h->d_rec_sys, n * (size_t)h->systems * sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return PCPD_OK;
}

int pcpd_paper_get_lattice(const pcpd_paper_t *h, uint32_t *host_out) {
  if (!h || !host_out) return fail(PCPD_EINVAL, "NULL argument");
  CU(cudaMemcpyAsync(host_out, h->d_lat, (size_t)h->systems * h->words * 4, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return PCPD_OK;
}

int pcpd_paper_set_lattice(pcpd_paper_t *h, const uint32_t *host_in, uint64_t step) {
  if (!h || !host_in) return fail(PCPD_EINVAL, "NULL argument");
  if (step > 0xFFFFFFFFull) return fail(PCPD_EINVAL, "step must be < 2^32");
  CU(cudaMemcpyAsync(h->d_lat, host_in, (size_t)h->systems * h->words * 4, cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->step = step;
  h->rec_steps.clear();
  if (h->d_rec_total) {
    CU(cudaMemsetAsync(h->d_rec_total, 0, h->rec_cap * sizeof(unsigned long long), h->stream));
    CU(cudaMemsetAsync(h->d_rec_sys, 0, h->rec_cap * (size_t)h->systems * sizeof(uint32_t), h->stream));
  }
  return PCPD_OK;
}

int pcpd_paper_get_plan(const pcpd_paper_t *h, uint32_t *systems_per_cta, uint32_t *threads,
                        uint32_t *grid, size_t *smem_bytes) {
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  if (systems_per_cta) *systems_per_cta = h->spc;
  if (threads) *threads = h->threads;
  if (grid) *grid = h->grid;
  if (smem_bytes) *smem_bytes = h->smem;
  return PCPD_OK;
}

int pcpd_paper_sync(pcpd_paper_t *h) {
  if (!h) return fail(PCPD_EINVAL, "NULL handle");
  CU(cudaStreamSynchronize(h->stream));
  return PCPD_OK;
}
