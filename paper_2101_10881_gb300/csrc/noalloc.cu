// noalloc.cu -- pes_eval_grad_static: evaluation and differentiation without
// any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's allocator or memory pool, plug-ins whose host forbids
// allocations on its device, or a path that must not change the device's
// memory footprint after start-up.  For them this entry point keeps everything
// the kernels need besides the caller's inputs and outputs -- job tables,
// completion flags, the control word and the workspace of forward, backward
// and cross products -- in one file-scope device array of a fixed size.  The
// array is part of the loaded library: every GPU that loads it holds it until
// the process exits.
//
// In host code the array's name is only a host-side stand-in; its device
// address is taken with cudaGetSymbolAddress (on the first call on a device,
// with that device current) and passed to the kernels.  The address belongs to
// the CUDA context the module was loaded into, so it is kept per device
// together with the identity of the context it was taken in: a call made in
// another context of the same device (a caller-created context, or the new
// primary context after cudaDeviceReset) takes the address again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pes.h"
#include "jobc.hpp"
#include "kernels.hpp"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
// the whole-series kernel only (no tiles): its shared-memory staging bounds the
// degree further at large k (471 at k=10, 543 at k=8, 839 at k=5, 991 at k=4)
constexpr int32_t kMaxStaticDegree = 1023;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
// per device: the array's address and the id of the context it was taken in
// (0: not taken yet, or the context could not be identified)
unsigned char* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

}  // namespace

namespace pes {
void set_last_error(const std::string& msg);
}

namespace {

void set_error(const std::string& msg) { pes::set_last_error(msg); }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Id of the current CUDA context (unique for the life of the process), 0 when
// the driver cannot tell; looked up through the runtime's driver entry points,
// so the library does not link the driver library itself.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_setup_mutex
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_static_scratch in the current context of the current
// device: taken with cudaGetSymbolAddress on the first call on that device
// (and again whenever the current context is not the one it was taken in, or
// the context cannot be identified).
pes_status setup_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return PES_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index out of range");
    return PES_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long ctx = current_context_id();  // 0 before the runtime made a context current
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = nullptr;
      g_scratch_ctx[dev] = 0;
      return PES_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    g_scratch_ctx[dev] = current_context_id();  // the context the address was taken in
  }
  *out = g_scratch_addr[dev];
  return PES_OK;
}

template <class T>
void put(std::vector<unsigned char>& blob, size_t off, const std::vector<T>& v) {
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
}

#define STATIC_CUDA(call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
      return PES_ECUDA;                                                      \
    }                                                                        \
  } while (0)

}  // namespace

extern "C" pes_status pes_eval_grad_static(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                                           int32_t d, int32_t k, const double* coeff, const double* input,
                                           double* value, double* grad, void* stream, int32_t* status_out) {
  if (!(k == 1 || k == 2 || k == 3 || k == 4 || k == 5 || k == 8 || k == 10)) {
    set_error("k must be one of 1,2,3,4,5,8,10");
    return PES_EUNSUPPORTED_K;
  }
  if (d < 0 || !coeff || !input || !value || !grad) {
    set_error("negative degree or NULL buffer");
    return PES_EINVAL;
  }
  if (d > kMaxStaticDegree) {
    set_error("degree " + std::to_string(d) + " above " + std::to_string(kMaxStaticDegree) +
              ", the largest the allocation-free entry point takes");
    return PES_EUNSUPPORTED_SIZE;
  }
  std::string msg = pes::validate(supp_ptr, supp_idx, N, n);
  if (!msg.empty()) {
    set_error(msg);
    return PES_EINVAL;
  }
  pes::Supports sup;
  sup.N = N;
  sup.n = n;
  if (N == 0) {
    sup.ptr.assign(1, 0);
  } else {
    sup.ptr.assign(supp_ptr, supp_ptr + N + 1);
    sup.idx.assign(supp_idx, supp_idx + sup.ptr.back());
  }
  const pes::Program1 G = pes::compile(sup, d, false, false);
  const int32_t S = pes::series_stride(d);
  const int64_t D1 = d + 1;

  // the integer pipe when the whole series of a job fit its staging (one lane
  // per coefficient pair within the CTA cap, shared memory within the opt-in
  // limit), else the FP64 pipe
  int dev = 0, nsm = 0, optin = 0;
  STATIC_CUDA(cudaGetDevice(&dev));
  STATIC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  STATIC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int arith = pes::ARITH_FP64;
  int threads = 128;
  {
    const int pairs = (d + 2) / 2;
    const int t = std::max((pairs + 31) / 32 * 32, std::min((2 * pairs + 31) / 32 * 32, pes::dag_max_threads(k)));
    if (t <= pes::dag_max_threads(k) &&
        pes::dag_smem_bytes(k, pes::ARITH_INT, S, d, 1, t) <= static_cast<size_t>(optin)) {
      arith = pes::ARITH_INT;
      threads = t;
    }
  }
  const int64_t sstride = pes::ws_slot_words(k, arith, S);

  // tables, in host memory first
  std::vector<pes::InstInfo> inst{{0, sstride, S, d}};
  std::vector<pes::CopyRow> rows;
  for (int32_t m = 0; m <= N; ++m) rows.push_back({m * D1, (N + 1) * D1, 0, 0, m, 0});
  for (int32_t i = 0; i < n; ++i) rows.push_back({i * D1, n * D1, 1, 0, 1 + N + i, 0});
  std::vector<pes::AddOut> outs;
  outs.push_back({0, D1, 0, 0, G.add_ptr[0], G.add_ptr[1]});
  for (int32_t i = 0; i < n; ++i) outs.push_back({i * D1, n * D1, 1, 0, G.add_ptr[1 + i], G.add_ptr[2 + i]});
  std::vector<int64_t> item_ptr(outs.size() + 1, 0);
  for (size_t o = 0; o < outs.size(); ++o) item_ptr[o + 1] = item_ptr[o] + D1;

  // layout inside the static array
  size_t off = 0;
  const size_t o_ctrl = off;
  off = align256(off + sizeof(pes::Ctrl));
  const size_t o_inst = off;
  off = align256(off + inst.size() * sizeof(pes::InstInfo));
  const size_t o_jobs = off;
  off = align256(off + G.jobs.size() * sizeof(pes::ConvJob));
  const size_t o_flags = off;
  off = align256(off + G.jobs.size() * sizeof(int32_t));
  const size_t o_rows = off;
  off = align256(off + rows.size() * sizeof(pes::CopyRow));
  const size_t o_outs = off;
  off = align256(off + outs.size() * sizeof(pes::AddOut));
  const size_t o_iptr = off;
  off = align256(off + item_ptr.size() * sizeof(int64_t));
  const size_t o_contrib = off;
  off = align256(off + G.add_src.size() * sizeof(int32_t));
  const size_t table_bytes = off;
  const size_t o_ws = off;
  const size_t ws_bytes = static_cast<size_t>(G.n_slots) * static_cast<size_t>(sstride) * sizeof(int32_t);
  if (o_ws + ws_bytes > kStaticScratchBytes) {
    set_error("problem needs " + std::to_string(o_ws + ws_bytes) + " bytes of scratch; the static array holds " +
              std::to_string(kStaticScratchBytes));
    return PES_EUNSUPPORTED_SIZE;
  }

  unsigned char* base = nullptr;
  pes_status s = setup_device(&base);
  if (s != PES_OK) return s;

  const size_t smem = pes::dag_smem_bytes(k, arith, S, d, 1, threads);
  if (smem > static_cast<size_t>(optin)) {
    set_error("degree " + std::to_string(d) + " at k=" + std::to_string(k) +
              " does not fit the shared-memory staging of whole series");
    return PES_EUNSUPPORTED_SIZE;
  }
  STATIC_CUDA(pes::dag_prepare(k, arith, smem));
  int per_sm = 0;
  STATIC_CUDA(pes::dag_occupancy(k, arith, threads, smem, &per_sm));
  if (per_sm < 1) {
    set_error("convolution kernel does not fit on an SM");
    return PES_EUNSUPPORTED_SIZE;
  }

  // every call starts from a zero control word and zero completion flags
  std::vector<unsigned char> blob(table_bytes, 0);
  put(blob, o_inst, inst);
  put(blob, o_jobs, G.jobs);
  put(blob, o_rows, rows);
  put(blob, o_outs, outs);
  put(blob, o_iptr, item_ptr);
  put(blob, o_contrib, G.add_src);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  STATIC_CUDA(cudaMemcpyAsync(base, blob.data(), table_bytes, cudaMemcpyHostToDevice, st));

  auto* ctrl = reinterpret_cast<pes::Ctrl*>(base + o_ctrl);
  auto* dinst = reinterpret_cast<pes::InstInfo*>(base + o_inst);
  int32_t* ws = reinterpret_cast<int32_t*>(base + o_ws);

  pes::CopyArgs ca{};
  ca.rows = reinterpret_cast<pes::CopyRow*>(base + o_rows);
  ca.nrows = static_cast<int32_t>(rows.size());
  ca.inst = dinst;
  ca.ws = ws;
  ca.src[0] = coeff;
  ca.src[1] = input;

  pes::DagArgs da{};
  da.jobs = reinterpret_cast<pes::ConvJob*>(base + o_jobs);
  da.njobs = static_cast<int32_t>(G.jobs.size());
  da.counter = 0;
  da.flags = reinterpret_cast<int32_t*>(base + o_flags);
  da.inst = dinst;
  da.ws = ws;
  da.ctrl = ctrl;
  da.smax = S;
  da.dmax = d;
  da.depth = 1;
  da.timeout_ns = 60000LL * 1000000LL;

  pes::AddArgs aa{};
  aa.outs = reinterpret_cast<pes::AddOut*>(base + o_outs);
  aa.nouts = static_cast<int32_t>(outs.size());
  aa.item_ptr = reinterpret_cast<int64_t*>(base + o_iptr);
  aa.contrib = reinterpret_cast<int32_t*>(base + o_contrib);
  aa.inst = dinst;
  aa.ws = ws;
  aa.dst[0] = value;
  aa.dst[1] = grad;
  int64_t maxc = 0;
  for (const auto& o : outs) maxc = std::max<int64_t>(maxc, o.cend - o.cbeg);
  aa.group_warps = pes::add_group_warps(maxc);

  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(static_cast<long long>(per_sm) * nsm,
                                                                               static_cast<long long>(da.njobs))));
  STATIC_CUDA(pes::launch_prologue(ctrl, st));
  STATIC_CUDA(pes::launch_pack(ca, k, arith, st));
  if (da.njobs > 0) STATIC_CUDA(pes::launch_dag(da, k, arith, threads, grid, st));
  STATIC_CUDA(pes::launch_add(aa, k, arith, item_ptr.back(), st));

  if (status_out) {
    STATIC_CUDA(cudaStreamSynchronize(st));
    int32_t dev_status = 0;
    STATIC_CUDA(cudaMemcpy(&dev_status, &ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    *status_out = dev_status;
  }
  return PES_OK;
}
