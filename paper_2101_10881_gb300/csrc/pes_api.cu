// pes_api.cu -- the C-ABI of include/pes.h: plans, batches and launches.
#include <cuda_runtime.h>

#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pes.h"
#include "jobc.hpp"
#include "kernels.hpp"

namespace {

thread_local std::string g_last_error;

pes_status fail(pes_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

pes_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return PES_ECUDA;
}

#define PES_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

bool valid_k(int32_t k) { return k == 1 || k == 2 || k == 3 || k == 4 || k == 5 || k == 8 || k == 10; }

template <class T>
pes_status upload(T** dptr, const std::vector<T>& v) {
  *dptr = nullptr;
  if (v.empty()) return PES_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dptr), v.size() * sizeof(T));
  if (e != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? fail(PES_ENOMEM, "device tables") : cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return PES_OK;
}

// One list of convolution jobs with its completion flags.
struct JobList {
  pes::ConvJob* jobs = nullptr;
  int32_t* flags = nullptr;
  int32_t n = 0;
  int32_t grid = 0;
  int32_t fparts = 1;  // parts per job the flags cover
};

// The outputs of an addition stage in two parts: those with at most 1,024
// contributions (one warp per output coefficient) and the longer sums (several
// warps per output coefficient, pes::add_group_warps); one launch per
// nonempty part, both reading the same contribution list.
struct AddTable {
  pes::AddOut* outs[2] = {nullptr, nullptr};
  int64_t* item_ptr[2] = {nullptr, nullptr};
  int32_t nouts[2] = {0, 0};
  int64_t items[2] = {0, 0};
  int32_t group_warps[2] = {1, 1};
  int32_t* contrib = nullptr;
  int32_t* mult = nullptr;  // integer factor per contribution (nullptr: all 1)
  int64_t total_items() const { return items[0] + items[1]; }
};

struct CopyTable {
  pes::CopyRow* rows = nullptr;
  int32_t n = 0;
};

// The arithmetic a launch shape uses: PES_ARITH_AUTO takes the integer pipe
// (whole series in shared memory where they fit, else output tiles).
int32_t resolve_arith(int32_t k, int32_t requested, int32_t dmax) {
  (void)k;
  (void)dmax;
  return requested != PES_ARITH_AUTO ? requested : pes::ARITH_INT;
}

// Threads per CTA of the whole-series kernel for the largest degree dmax
// (`requested` 0: automatic), or 0 when no CTA shape within the cap holds one
// lane per coefficient pair (integer variant).
int32_t whole_series_threads(int32_t k, int32_t arith, int32_t dmax, int32_t requested) {
  int32_t t = requested;
  if (arith == pes::ARITH_INT) {
    // by default two lanes per coefficient pair (one per output coefficient),
    // three at k = 10 (whose CTAs are capped at 256 threads and two per SM:
    // the wider CTA keeps 16 warps per SM where its exchange rows allow two),
    // whole warps; at least one lane per pair
    const int32_t pairs = (dmax + 2) / 2;
    const int32_t least = (pairs + 31) / 32 * 32;
    const int32_t per_pair = k >= 10 ? 3 : 2;
    t = t == 0 ? std::max(least, std::min((per_pair * pairs + 31) / 32 * 32, pes::dag_max_threads(k)))
               : std::max(t, least);
  } else if (t == 0) {
    t = 128;  // FP64 variant: 128 threads share the terms evenly
  }
  return t <= pes::dag_max_threads(k) ? t : 0;
}

// The whole-series kernel runs degree dmax (lanes and shared memory at staging
// depth 1); otherwise the tiled kernel takes it.
bool whole_series_fits(int32_t k, int32_t arith, int32_t dmax, int32_t requested, int optin) {
  const int32_t t = whole_series_threads(k, arith, dmax, requested);
  return t > 0 && pes::dag_smem_bytes(k, arith, pes::series_stride(dmax), dmax, 1, t) <= static_cast<size_t>(optin);
}

int device_optin() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return optin;
}

// Device state shared by single plans and batches.

struct Exec {
  int32_t k = 0, arith = 0, threads = 128, ctas_per_sm = 0;
  int32_t smax = 0, dmax = 0;
  int32_t depth = 1, staging = 0;  // staging depth in use; requested (0 = automatic)
  int32_t split = 1, split_req = 0;  // parts per convolution job in use; requested (0 = automatic)
  int32_t tile = 0;  // > 0: the tiled kernel, output tiles of this many coefficients (split = tiles per job)
  size_t smem = 0;
  int32_t blocks_per_sm = 0, nsm = 0, optin = 0;
  long long timeout_ns = 0;
  pes::InstInfo* inst = nullptr;
  pes::Ctrl* ctrl = nullptr;
  int32_t* ws = nullptr;  // every series in digit form (see pes::InstInfo)
  size_t ws_words = 0;
  std::vector<void*> owned;
  // profiling: events around the phases of the last call
  bool profile = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int32_t last_launches = 0;
  bool has_unpack = false;

  ~Exec() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (void* p : owned) cudaFree(p);
    cudaFree(inst);
    cudaFree(ctrl);
    cudaFree(ws);
  }

  template <class T>
  pes_status put(T** dptr, const std::vector<T>& v) {
    pes_status s = upload(dptr, v);
    if (s == PES_OK && *dptr) owned.push_back(*dptr);
    return s;
  }

  // Parts per job when the caller left it automatic (integer pipe, whole
  // series): a table whose layers hold few jobs for the CTAs of the launch
  // (one polynomial of few long monomials, one rank's share of a polynomial)
  // runs its dependency chains faster with every job split over several CTAs.
  // The parts double while the average layer, times the parts, holds fewer
  // sub-jobs than the launch has CTAs and every part keeps at least 8
  // coefficient pairs (measured on the p2-like polynomial at d=152, k=10:
  // within 10 % of the best split for 1 to 128 monomials).
  void choose_split(const std::vector<pes::ConvJob>& jobs) {
    if (split_req != 0 || arith != pes::ARITH_INT || tile != 0 || jobs.empty()) return;
    int32_t lo = jobs.front().layer, hi = jobs.front().layer;
    for (const auto& j : jobs) {
      lo = std::min(lo, j.layer);
      hi = std::max(hi, j.layer);
    }
    const double width = static_cast<double>(jobs.size()) / (hi - lo + 1);
    const double ctas = static_cast<double>(blocks_per_sm) * nsm;
    const int32_t most = std::max(1, (dmax + 2) / 2 / 8);
    int32_t sp = 1;
    while (sp < pes::kMaxSplit && 2 * sp <= most && width * sp < ctas) sp *= 2;
    split = sp;
  }

  // Parts per job the flags of a job list must cover: the split in use, and,
  // when the split is automatic, every split the autotuner may try (1, 2 and
  // half to twice the automatic choice); the tiled kernel flags every tile.
  int32_t flag_parts() const {
    if (tile > 0 || split_req != 0 || arith != pes::ARITH_INT) return std::max(split, 1);
    return std::max(2, std::min(pes::kMaxSplit, 2 * split));
  }

  pes_status make_joblist(JobList& L, const std::vector<pes::ConvJob>& jobs) {
    L.n = static_cast<int32_t>(jobs.size());
    pes_status s = put(&L.jobs, jobs);
    if (s != PES_OK) return s;
    if (L.n > 0) {
      // one flag per part of every job (tiled kernel: per tile)
      if (static_cast<int64_t>(L.n) * flag_parts() >= (1LL << 31))
        return fail(PES_EUNSUPPORTED_SIZE, "jobs x tiles per job exceed 2^31");
      L.fparts = flag_parts();
      const size_t nf = static_cast<size_t>(L.n) * L.fparts;
      cudaError_t e = cudaMalloc(&L.flags, sizeof(int32_t) * nf);
      if (e != cudaSuccess) return fail(PES_ENOMEM, "job flags");
      owned.push_back(L.flags);
      PES_CUDA(cudaMemset(L.flags, 0, sizeof(int32_t) * nf));
    }
    long long cap = static_cast<long long>(blocks_per_sm) * nsm;
    L.grid = static_cast<int32_t>(
        std::max<long long>(1, std::min<long long>(cap, static_cast<long long>(L.n) * split)));
    return PES_OK;
  }

  // mult: integer factor of every contribution, or empty when all are 1
  pes_status make_add(AddTable& A, const std::vector<pes::AddOut>& outs, const std::vector<int32_t>& contrib,
                      const std::vector<pes::InstInfo>& insts, const std::vector<int32_t>& mult = {}) {
    std::vector<pes::AddOut> part[2];
    int64_t maxc[2] = {0, 0};
    for (const auto& o : outs) {
      const int64_t c = o.cend - o.cbeg;
      const int b = pes::add_group_warps(c) > 1 ? 1 : 0;
      part[b].push_back(o);
      maxc[b] = std::max(maxc[b], c);
    }
    pes_status s = PES_OK;
    for (int b = 0; b < 2 && s == PES_OK; ++b) {
      A.nouts[b] = static_cast<int32_t>(part[b].size());
      std::vector<int64_t> ip(part[b].size() + 1, 0);
      for (size_t o = 0; o < part[b].size(); ++o)
        ip[o + 1] = ip[o] + insts[static_cast<size_t>(part[b][o].inst)].d + 1;
      A.items[b] = ip.back();
      A.group_warps[b] = pes::add_group_warps(maxc[b], A.items[b], nsm > 0 ? nsm : 1);
      if (!part[b].empty()) {
        s = put(&A.outs[b], part[b]);
        if (s == PES_OK) s = put(&A.item_ptr[b], ip);
      }
    }
    if (s == PES_OK) s = put(&A.contrib, contrib);
    const bool ones = std::all_of(mult.begin(), mult.end(), [](int32_t v) { return v == 1; });
    if (s == PES_OK && !ones) s = put(&A.mult, mult);
    return s;
  }

  // `o.arith` must be resolved (resolve_arith) before the instances' workspace
  // offsets are laid out: the words per series depend on the arithmetic.
  pes_status init(int32_t k_, const pes_options& o, const std::vector<pes::InstInfo>& insts, size_t ws_words_) {
    k = k_;
    arith = o.arith;
    threads = o.threads;
    ctas_per_sm = o.ctas_per_sm;
    timeout_ns = (o.timeout_ms > 0 ? o.timeout_ms : 60000) * 1000000LL;
    smax = 8;
    dmax = 0;
    for (const auto& in : insts) {
      smax = std::max(smax, in.S);
      dmax = std::max(dmax, in.d);
    }
    int dev = 0;
    PES_CUDA(cudaGetDevice(&dev));
    PES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PES_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    staging = o.staging;
    split_req = o.split;
    if (o.tile == 0 && whole_series_fits(k, arith, dmax, threads, optin)) {
      // whole series in shared memory; staging depth 2 only when asked for and
      // it fits (the autotuner tries both)
      tile = 0;
      threads = whole_series_threads(k, arith, dmax, threads);
      split = (arith == pes::ARITH_INT && o.split > 0) ? o.split : 1;
      depth = (staging == 2 && pes::dag_smem_bytes(k, arith, smax, dmax, 2, threads) <= static_cast<size_t>(optin))
                  ? 2
                  : 1;
      smem = pes::dag_smem_bytes(k, arith, smax, dmax, depth, threads);
    } else {
      // output tiles: at least one lane per pair of coefficients of a tile; by
      // default two per pair (integer variant) or 128 threads (FP64 variant)
      tile = o.tile > 0 ? o.tile : pes::kDefaultTile;
      if (threads == 0)
        threads = arith == pes::ARITH_INT ? std::min(2 * tile, pes::dag_max_threads(k)) : 128;
      threads = std::max(threads, (tile / 2 + 31) / 32 * 32);
      if (threads > pes::dag_max_threads(k))
        return fail(PES_EUNSUPPORTED_SIZE, "tiles of " + std::to_string(tile) + " coefficients need " +
                                               std::to_string(threads) + " threads per CTA; at most " +
                                               std::to_string(pes::dag_max_threads(k)) + " at k=" + std::to_string(k));
      split = (dmax + tile) / tile;
      depth = 1;
      smem = pes::dag_tiled_smem_bytes(k, arith, tile);
    }
    if (smem > static_cast<size_t>(optin))
      return fail(PES_EUNSUPPORTED_SIZE, "degree " + std::to_string(dmax) + " needs " + std::to_string(smem) +
                                             " bytes of shared memory at k=" + std::to_string(k));
    PES_CUDA(pes::dag_prepare(k, arith, smem, tile > 0));
    PES_CUDA(pes::dag_occupancy(k, arith, threads, smem, &blocks_per_sm, tile > 0));
    if (blocks_per_sm < 1) return fail(PES_EUNSUPPORTED_SIZE, "convolution kernel does not fit on an SM");
    if (ctas_per_sm > 0) blocks_per_sm = std::min(blocks_per_sm, ctas_per_sm);
    pes_status s = upload(&inst, insts);
    if (s != PES_OK) return s;
    cudaError_t e = cudaMalloc(&ctrl, sizeof(pes::Ctrl));
    if (e != cudaSuccess) return fail(PES_ENOMEM, "control block");
    PES_CUDA(cudaMemset(ctrl, 0, sizeof(pes::Ctrl)));
    profile = o.profile != 0;
    if (profile)
      for (cudaEvent_t& e : ev) PES_CUDA(cudaEventCreate(&e));
    ws_words = std::max<size_t>(ws_words_, 8);
    e = cudaMalloc(&ws, ws_words * sizeof(int32_t));
    if (e != cudaSuccess) return fail(PES_ENOMEM, "workspace of " + std::to_string(ws_words * 4) + " bytes");
    PES_CUDA(cudaMemset(ws, 0, ws_words * sizeof(int32_t)));
    return PES_OK;
  }

  // shared memory of the convolution kernel at staging depth `dp` with `t`
  // threads per CTA, or 0 if it does not fit
  size_t smem_at(int32_t dp, int32_t t) const {
    if (tile > 0) return dp == 1 ? pes::dag_tiled_smem_bytes(k, arith, tile) : 0;
    const size_t b = pes::dag_smem_bytes(k, arith, smax, dmax, dp, t);
    return b <= static_cast<size_t>(optin) ? b : 0;
  }

  // threads per CTA, a cap on CTAs per SM (0: as many as fit), the staging
  // depth and the parts per job (integer variant only; the tiled kernel keeps
  // its tiles per job) for later launches
  pes_status configure(int32_t t, int32_t ctas_cap, int32_t dp, int32_t sp, JobList& L) {
    const size_t b = smem_at(dp, t);
    if (b == 0) return fail(PES_EUNSUPPORTED_SIZE, "staging depth does not fit in shared memory");
    if (tile > 0 && t < tile / 2) return fail(PES_EUNSUPPORTED_SIZE, "fewer lanes than pairs of a tile");
    if (tile == 0 && arith == pes::ARITH_INT && L.n > 0 && std::max(1, sp) > L.fparts)
      return fail(PES_EINTERNAL, "parts per job beyond the job flags");
    PES_CUDA(pes::dag_prepare(k, arith, b, tile > 0));
    int bps = 0;
    PES_CUDA(pes::dag_occupancy(k, arith, t, b, &bps, tile > 0));
    if (bps < 1) return fail(PES_EUNSUPPORTED_SIZE, "configuration does not fit on an SM");
    smem = b;
    depth = dp;
    if (tile == 0) split = arith == pes::ARITH_INT ? std::max(1, sp) : 1;
    threads = t;
    blocks_per_sm = ctas_cap > 0 ? std::min(bps, ctas_cap) : bps;
    L.grid = static_cast<int32_t>(std::max<long long>(1, std::min<long long>(
                 static_cast<long long>(blocks_per_sm) * nsm, static_cast<long long>(L.n) * split)));
    return PES_OK;
  }

  pes::DagArgs dag_args(const JobList& L, int counter) const {
    pes::DagArgs a{};
    a.jobs = L.jobs;
    a.njobs = L.n;
    a.counter = counter;
    a.flags = L.flags;
    a.inst = inst;
    a.ws = ws;
    a.ctrl = ctrl;
    a.smax = smax;
    a.dmax = dmax;
    a.depth = depth;
    a.split = split;
    a.timeout_ns = timeout_ns;
    a.tile = tile;
    return a;
  }

  cudaError_t run_dag(const JobList& L, int counter, cudaStream_t st) const {
    if (L.n == 0) return cudaSuccess;
    return pes::launch_dag(dag_args(L, counter), k, arith, threads, L.grid, st);
  }

  // sums into caller buffers (rounded to k limbs), or, with dst0 == dst1 ==
  // nullptr, into workspace slots in digit form
  cudaError_t run_add(const AddTable& A, double* dst0, double* dst1, cudaStream_t st, int32_t mode = 0,
                      int32_t* grid_io = nullptr, long long* acc_out = nullptr) const {
    pes::AddArgs args[2]{};
    for (int b = 0; b < 2; ++b) {
      if (A.items[b] == 0) continue;
      pes::AddArgs& a = args[b];
      a.mode = mode;
      a.grid_io = grid_io;
      a.acc_out = acc_out;
      a.outs = A.outs[b];
      a.nouts = A.nouts[b];
      a.to_ws = (dst0 == nullptr && dst1 == nullptr) ? 1 : 0;
      a.item_ptr = A.item_ptr[b];
      a.contrib = A.contrib;
      a.mult = A.mult;
      a.inst = inst;
      a.ws = ws;
      a.dst[0] = dst0;
      a.dst[1] = dst1;
      a.group_warps = A.group_warps[b];
    }
    if (paired(A)) return pes::launch_add_pair(args[0], A.items[0], args[1], A.items[1], k, arith, st);
    for (int b = 0; b < 2; ++b) {
      if (A.items[b] == 0) continue;
      cudaError_t e = pes::launch_add(args[b], k, arith, A.items[b], st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // both parts of an addition stage in one launch (both summed by warp groups)
  static bool paired(const AddTable& A) {
    return A.items[0] > 0 && A.items[1] > 0 && A.group_warps[0] > 1 && A.group_warps[1] > 1;
  }

  // kernels a run_add / run_dag / run_pack / run_unpack call launches
  static int32_t launches(const AddTable& A) { return paired(A) ? 1 : (A.items[0] > 0) + (A.items[1] > 0); }
  static int32_t launches(const JobList& L) { return L.n > 0 ? 1 : 0; }
  static int32_t launches(const CopyTable& C) { return C.n > 0 ? 1 : 0; }

  cudaError_t run_pack(const CopyTable& C, const double* s0, const double* s1, const double* s2,
                       cudaStream_t st) const {
    pes::CopyArgs a{};
    a.rows = C.rows;
    a.nrows = C.n;
    a.inst = inst;
    a.ws = ws;
    a.src[0] = s0;
    a.src[1] = s1;
    a.src[2] = s2;
    return pes::launch_pack(a, k, arith, st);
  }

  cudaError_t run_unpack(const CopyTable& C, double* d0, double* d1, cudaStream_t st) const {
    pes::CopyArgs a{};
    a.rows = C.rows;
    a.nrows = C.n;
    a.inst = inst;
    a.ws = ws;
    a.dst[0] = d0;
    a.dst[1] = d1;
    return pes::launch_unpack(a, k, arith, st);
  }

  // record phase boundary i (0..4) of the current call
  cudaError_t mark(int i, cudaStream_t st) const { return profile ? cudaEventRecord(ev[i], st) : cudaSuccess; }

  pes_status last_timing(double* ms, int32_t* launches) {
    if (!profile) return fail(PES_EINVAL, "built without profile = 1");
    PES_CUDA(cudaEventSynchronize(ev[4]));
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      PES_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      if (ms) ms[i] = t;
    }
    if (launches) *launches = last_launches;
    return PES_OK;
  }

  pes_status check(cudaStream_t st) {
    PES_CUDA(cudaStreamSynchronize(st));
    pes::Ctrl h{};
    PES_CUDA(cudaMemcpy(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.status != 0) {
      int32_t zero[3] = {h.epoch, 0, 0};
      PES_CUDA(cudaMemcpy(ctrl, zero, sizeof(zero), cudaMemcpyHostToDevice));
      g_last_error = "device wait gave up: job " + std::to_string(h.diag[1]) + " waiting on " +
                     std::to_string(h.diag[0]);
      return static_cast<pes_status>(h.status);
    }
    return PES_OK;
  }
};

pes_status parse_options(const pes_options* opt, pes_options& o) {
  pes_default_options(&o);
  if (opt) o = *opt;
  if (o.arith != PES_ARITH_AUTO && o.arith != PES_ARITH_FP64 && o.arith != PES_ARITH_INT)
    return fail(PES_EINVAL, "arith must be -1, 0 or 1");
  if (o.threads < 0 || o.threads > 1024 || o.threads % 32 != 0)
    return fail(PES_EINVAL, "threads must be 0 (automatic) or a multiple of 32 up to 1024");
  if (o.ctas_per_sm < 0) return fail(PES_EINVAL, "ctas_per_sm must be >= 0");
  if (o.staging < 0 || o.staging > 2) return fail(PES_EINVAL, "staging must be 0, 1 or 2");
  if (!(o.split == 0 || o.split == 1 || o.split == 2 || o.split == 4 || o.split == 8 || o.split == 16))
    return fail(PES_EINVAL, "split must be 0, 1, 2, 4, 8 or 16");
  if (o.tile != 0 && (o.tile < 16 || o.tile > 1024 || o.tile % 8 != 0))
    return fail(PES_EINVAL, "tile must be 0 (automatic) or a multiple of 8 in [16, 1024]");
  return PES_OK;
}

pes_status build_supports(const int32_t* ptr, const int32_t* idx, int32_t N, int32_t n, pes::Supports& s,
                          const int32_t* ex = nullptr) {
  std::string msg = pes::validate(ptr, idx, N, n);
  if (!msg.empty()) return fail(PES_EINVAL, msg);
  msg = pes::validate_exponents(ptr, ex, N);
  if (!msg.empty()) return fail(PES_EINVAL, msg);
  s.N = N;
  s.n = n;
  if (N == 0) {
    s.ptr.assign(1, 0);
    s.idx.clear();
    s.ex.clear();
  } else {
    s.ptr.assign(ptr, ptr + (N + 1));
    s.idx.assign(idx, idx + s.ptr.back());
    if (ex != nullptr && std::any_of(ex, ex + s.ptr.back(), [](int32_t e) { return e != 1; }))
      s.ex.assign(ex, ex + s.ptr.back());
    else
      s.ex.clear();
  }
  return PES_OK;
}

// Dependencies of a job list taken out of a larger one: an operand produced by
// an earlier job of the list waits for it; any other operand is already in
// the workspace.
void resolve_local_deps(std::vector<pes::ConvJob>& jobs) {
  std::map<int32_t, int32_t> producer;
  for (size_t j = 0; j < jobs.size(); ++j) {
    auto p1 = producer.find(jobs[j].in1), p2 = producer.find(jobs[j].in2);
    jobs[j].dep1 = p1 == producer.end() ? -1 : p1->second;
    jobs[j].dep2 = p2 == producer.end() ? -1 : p2->second;
    producer[jobs[j].out] = static_cast<int32_t>(j);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// autotuning of the convolution launch shape
// ---------------------------------------------------------------------------

namespace {

void fnv_mix(uint64_t& h, int64_t v) {
  for (int i = 0; i < 8; ++i) {
    h ^= static_cast<uint64_t>((v >> (8 * i)) & 0xFF);
    h *= 1099511628211ull;
  }
}

std::string autotune_cache_file() {
  const char* p = std::getenv("PES_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/pes_autotune.txt";
}

bool tune_lookup(const std::string& key, int32_t* threads, int32_t* ctas, int32_t* depth, int32_t* split) {
  FILE* f = std::fopen(autotune_cache_file().c_str(), "r");
  if (!f) return false;
  char line[512], kb[256];
  int t = 0, c = 0, dp = 0, sp = 0;
  bool found = false;
  while (std::fgets(line, sizeof(line), f))
    if (std::sscanf(line, "%255s %d %d %d %d", kb, &t, &c, &dp, &sp) == 5 && key == kb) {
      *threads = t;
      *ctas = c;
      *depth = dp;
      *split = sp;
      found = true;
    }
  std::fclose(f);
  return found;
}

void tune_store(const std::string& key, int32_t threads, int32_t ctas, int32_t depth, int32_t split) {
  const std::string path = autotune_cache_file();
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos)
    for (size_t i = 1; i <= slash; ++i)
      if (i == slash || path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), threads, ctas, depth, split);
  std::fclose(f);
}

// Time `run` (one whole call on `st`) for every candidate launch shape of the
// convolution kernel and keep the fastest; the values do not depend on the
// shape, so the trials may run on the caller's data.  Cached by `key`.
template <class Run>
pes_status tune_launch(Exec& E, JobList& L, const std::string& key, Run run, cudaStream_t st) {
  int32_t bt = E.threads, bc = 0, bd = E.depth, bs = E.split;
  if (!tune_lookup(key, &bt, &bc, &bd, &bs)) {
    const int32_t base = E.threads;
    std::vector<int32_t> ts{base};
    if (E.arith == pes::ARITH_INT) {
      for (int32_t t : {base + 32, (base * 3 / 2 + 31) / 32 * 32, base * 2})
        if (t <= pes::dag_max_threads(E.k) && std::find(ts.begin(), ts.end(), t) == ts.end()) ts.push_back(t);
    } else {
      ts.push_back(256);
    }
    std::vector<int32_t> depths{E.depth};
    if (E.staging == 0) depths = {1, 2};
    std::vector<int32_t> splits{E.split};
    if (E.split_req == 0 && E.arith == pes::ARITH_INT && E.tile == 0) {
      // the automatic choice (E.split), half and twice it, and 1 and 2
      splits = {1, 2};
      for (int32_t sp : {E.split / 2, E.split, E.split * 2})
        if (sp >= 1 && sp <= pes::kMaxSplit && std::find(splits.begin(), splits.end(), sp) == splits.end())
          splits.push_back(sp);
    }
    cudaEvent_t e0, e1;
    PES_CUDA(cudaEventCreate(&e0));
    PES_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int32_t sp : splits) {
      for (int32_t dp : depths) {
        for (int32_t t : ts) {
          const size_t b = E.smem_at(dp, t);
          if (b == 0) continue;
          PES_CUDA(pes::dag_prepare(E.k, E.arith, b));
          int occ = 0;
          PES_CUDA(pes::dag_occupancy(E.k, E.arith, t, b, &occ));
          for (int32_t c = std::max(1, occ); c >= std::max(1, occ - 1); --c) {
            pes_status s = E.configure(t, c, dp, sp, L);
            if (s != PES_OK) continue;
            s = run(st);  // warm-up
            if (s != PES_OK) return s;
            PES_CUDA(cudaEventRecord(e0, st));
            s = run(st);
            if (s != PES_OK) return s;
            PES_CUDA(cudaEventRecord(e1, st));
            PES_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            PES_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
              best = ms;
              bt = t;
              bc = c;
              bd = dp;
              bs = sp;
            }
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, bt, bc, bd, bs);
  }
  return E.configure(bt, bc, bd, bs, L);
}

std::string tune_key(const Exec& E, int64_t njobs, uint64_t signature) {
  char key[200];
  std::snprintf(key, sizeof(key), "v6_k%d_a%d_t%d_s%d_p%d_T%d_d%d_j%lld_%016llx", E.k, E.arith, E.threads,
                E.staging, E.split_req, E.tile, E.dmax,
                static_cast<long long>(njobs), static_cast<unsigned long long>(signature));
  return key;
}

}  // namespace

// ---------------------------------------------------------------------------
// single plans
// ---------------------------------------------------------------------------

struct pes_plan_s {
  pes::Program1 prog;
  Exec ex;
  bool autotune = false, tuned = false;
  uint64_t signature = 1469598103934665603ull;
  JobList fwd, vjp_fwd, vjp_m, vjp_corr;
  AddTable add, add_g;
  CopyTable pack, pack_u, unpack;
  bool with_vjp = false;
  bool complex_series = false;
  AddTable add_mat;  // systems: values and Jacobian with one P x n matrix per power of t
  AddTable add_gi;   // systems: grad_input[i] = sum over the polynomials of the correlations
  int64_t ws_bytes = 0;
};

extern "C" void pes_default_options(pes_options* opt) {
  if (!opt) return;
  opt->arith = PES_ARITH_AUTO;
  opt->threads = 0;
  opt->ctas_per_sm = 0;
  opt->with_vjp = 1;
  opt->timeout_ms = 60000;
  opt->profile = 0;
  opt->autotune = 0;
  opt->staging = 0;
  opt->split = 0;
  opt->tile = 0;
}

extern "C" pes_status pes_plan(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n, int32_t d,
                               int32_t k, pes_plan_t* out) {
  return pes_plan_ex(supp_ptr, supp_idx, N, n, d, k, nullptr, out);
}

namespace {
pes_status plan_impl(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N, int32_t n,
                     int32_t d, int32_t k, const pes_options* opt, pes_plan_t* out, bool complex_series = false,
                     const std::vector<int32_t>* poly_ptr = nullptr);
}  // namespace

extern "C" pes_status pes_plan_ex(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n, int32_t d,
                                  int32_t k, const pes_options* opt, pes_plan_t* out) {
  return plan_impl(supp_ptr, supp_idx, nullptr, N, n, d, k, opt, out);
}

extern "C" pes_status pes_plan_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                      int32_t N, int32_t n, int32_t d, int32_t k, const pes_options* opt,
                                      pes_plan_t* out) {
  if (!supp_exp && N > 0) return fail(PES_EINVAL, "supp_exp is NULL");
  return plan_impl(supp_ptr, supp_idx, supp_exp, N, n, d, k, opt, out);
}

extern "C" pes_status pes_plan_complex(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                       int32_t N, int32_t n, int32_t d, int32_t k, const pes_options* opt,
                                       pes_plan_t* out) {
  return plan_impl(supp_ptr, supp_idx, supp_exp, N, n, d, k, opt, out, true);
}

extern "C" pes_status pes_plan_system(int32_t P, const int32_t* poly_ptr, const int32_t* supp_ptr,
                                      const int32_t* supp_idx, const int32_t* supp_exp, int32_t n, int32_t d,
                                      int32_t k, const pes_options* opt, pes_plan_t* out) {
  if (P < 1 || !poly_ptr) return fail(PES_EINVAL, "a system needs P >= 1 polynomials and poly_ptr");
  if (n < 1 || static_cast<int64_t>(P) * (n + 1) >= (1LL << 30))
    return fail(PES_EINVAL, "P x (n + 1) outputs must stay below 2^30");
  if (poly_ptr[0] != 0) return fail(PES_EINVAL, "poly_ptr[0] must be 0");
  for (int32_t p = 0; p < P; ++p)
    if (poly_ptr[p + 1] < poly_ptr[p]) return fail(PES_EINVAL, "poly_ptr must not decrease");
  std::vector<int32_t> pp(poly_ptr, poly_ptr + P + 1);
  return plan_impl(supp_ptr, supp_idx, supp_exp, poly_ptr[P], n, d, k, opt, out, false, &pp);
}

namespace {
pes_status plan_impl(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp, int32_t N, int32_t n,
                     int32_t d, int32_t k, const pes_options* opt, pes_plan_t* out, bool complex_series,
                     const std::vector<int32_t>* poly_ptr) {
  if (!out) return fail(PES_EINVAL, "out is NULL");
  *out = nullptr;
  if (!valid_k(k)) return fail(PES_EUNSUPPORTED_K, "k must be one of 1,2,3,4,5,8,10");
  if (d < 0) return fail(PES_EINVAL, "d must be >= 0");
  if (d > pes::kMaxDegree) return fail(PES_EUNSUPPORTED_SIZE, "d must be <= " + std::to_string(pes::kMaxDegree));
  pes_options o;
  pes_status s = parse_options(opt, o);
  if (s != PES_OK) return s;
  pes::Supports sup;
  s = build_supports(supp_ptr, supp_idx, N, n, sup, supp_exp);
  if (s != PES_OK) return s;

  std::unique_ptr<pes_plan_s> P(new (std::nothrow) pes_plan_s());
  if (!P) return fail(PES_ENOMEM, "plan");
  P->with_vjp = o.with_vjp != 0;
  P->complex_series = complex_series;
  if (poly_ptr != nullptr) {
    P->prog = pes::compile_system(sup, *poly_ptr, d, P->with_vjp);
  } else {
    P->prog = pes::compile(sup, d, false, P->with_vjp);
    if (complex_series) P->prog = pes::complexify(P->prog);
  }
  const pes::Program1& G = P->prog;
  const int32_t S = pes::series_stride(d);
  const int32_t slots = P->with_vjp ? G.n_slots_vjp : G.n_slots;
  o.arith = resolve_arith(k, o.arith, d);
  const int64_t sstride = pes::ws_slot_words(k, o.arith, S);
  std::vector<pes::InstInfo> insts{{0, sstride, S, d}};
  s = P->ex.init(k, o, insts, static_cast<size_t>(slots) * static_cast<size_t>(sstride));
  if (s != PES_OK) return s;
  P->ws_bytes = static_cast<int64_t>(P->ex.ws_words * sizeof(int32_t));

  // forward jobs
  P->ex.choose_split(G.jobs);
  s = P->ex.make_joblist(P->fwd, G.jobs);
  if (s != PES_OK) return s;
  P->autotune = o.autotune != 0;
  for (const auto& j : G.jobs) {
    fnv_mix(P->signature, j.layer);
    fnv_mix(P->signature, j.dep1);
    fnv_mix(P->signature, j.dep2);
  }

  // pack rows: coefficients (buffer 0), inputs (buffer 1); complex series: the
  // real part from the first block of the buffer, the imaginary part from the
  // second, into slots 2s and 2s + 1
  const int64_t D1 = d + 1;
  const int64_t cim = static_cast<int64_t>(k) * (N + 1) * D1, iim = static_cast<int64_t>(k) * n * D1;
  std::vector<pes::CopyRow> rows;
  const int32_t np = G.system_P;
  if (np > 0) {
    // system: coefficient series of polynomial p at (its constant, its monomials),
    // consecutive: constant at poly_ptr[p] + p, monomial m at m + p + 1
    const int64_t cl = static_cast<int64_t>(N + np) * D1;
    for (int32_t p = 0; p < np; ++p) {
      const int32_t m0 = (*poly_ptr)[static_cast<size_t>(p)], m1 = (*poly_ptr)[static_cast<size_t>(p) + 1];
      rows.push_back({static_cast<int64_t>(m0 + p) * D1, cl, 0, 0, G.const0 + p, 0});
      for (int32_t m = m0; m < m1; ++m) rows.push_back({static_cast<int64_t>(m + p + 1) * D1, cl, 0, 0, m + 1, 0});
    }
    for (int32_t i = 0; i < n; ++i) rows.push_back({i * D1, n * D1, 1, 0, 1 + N + i, 0});
  } else if (!complex_series) {
    for (int32_t m = 0; m <= N; ++m) rows.push_back({m * D1, (N + 1) * D1, 0, 0, m, 0});
    for (int32_t i = 0; i < n; ++i) rows.push_back({i * D1, n * D1, 1, 0, 1 + N + i, 0});
  } else {
    for (int32_t m = 0; m <= N; ++m) {
      rows.push_back({m * D1, (N + 1) * D1, 0, 0, 2 * m, 0});
      rows.push_back({cim + m * D1, (N + 1) * D1, 0, 0, 2 * m + 1, 0});
    }
    for (int32_t i = 0; i < n; ++i) {
      rows.push_back({i * D1, n * D1, 1, 0, 2 * (1 + N + i), 0});
      rows.push_back({iim + i * D1, n * D1, 1, 0, 2 * (1 + N + i) + 1, 0});
    }
  }
  P->pack.n = static_cast<int32_t>(rows.size());
  s = P->ex.put(&P->pack.rows, rows);
  if (s != PES_OK) return s;

  // addition: value (buffer 0) and gradients (buffer 1); complex series: output
  // 2o the real part (first block), 2o + 1 the imaginary part (second block)
  std::vector<pes::AddOut> outs;
  if (np > 0) {
    // system: values [k][P][d+1] (buffer 0), Jacobian [k][P][n][d+1] (buffer 1);
    // and the same sums into one P-vector / P x n matrix per power of t
    // ([k][d+1][P], [k][d+1][P][n]) for pes_eval_system's matrix layout
    std::vector<pes::AddOut> mat;
    for (int32_t p = 0; p < np; ++p) {
      outs.push_back({p * D1, np * D1, 0, 0, G.add_ptr[static_cast<size_t>(p)], G.add_ptr[static_cast<size_t>(p) + 1]});
      mat.push_back({p, D1 * np, 0, 0, G.add_ptr[static_cast<size_t>(p)], G.add_ptr[static_cast<size_t>(p) + 1], np});
    }
    for (int32_t p = 0; p < np; ++p)
      for (int32_t i = 0; i < n; ++i) {
        const size_t o = static_cast<size_t>(np + p * n + i);
        outs.push_back({static_cast<int64_t>(p * n + i) * D1, static_cast<int64_t>(np) * n * D1, 1, 0,
                        G.add_ptr[o], G.add_ptr[o + 1]});
        mat.push_back({static_cast<int64_t>(p) * n + i, D1 * np * n, 1, 0, G.add_ptr[o], G.add_ptr[o + 1],
                       static_cast<int64_t>(np) * n});
      }
    s = P->ex.make_add(P->add_mat, mat, G.add_src, insts, G.add_mult);
    if (s != PES_OK) return s;
  } else if (!complex_series) {
    outs.push_back({0, D1, 0, 0, G.add_ptr[0], G.add_ptr[1]});
    for (int32_t i = 0; i < n; ++i) outs.push_back({i * D1, n * D1, 1, 0, G.add_ptr[1 + i], G.add_ptr[2 + i]});
  } else {
    const int64_t vim = static_cast<int64_t>(k) * D1;
    outs.push_back({0, D1, 0, 0, G.add_ptr[0], G.add_ptr[1]});
    outs.push_back({vim, D1, 0, 0, G.add_ptr[1], G.add_ptr[2]});
    for (int32_t i = 0; i < n; ++i) {
      outs.push_back({i * D1, n * D1, 1, 0, G.add_ptr[2 + 2 * i], G.add_ptr[3 + 2 * i]});
      outs.push_back({iim + i * D1, n * D1, 1, 0, G.add_ptr[3 + 2 * i], G.add_ptr[4 + 2 * i]});
    }
  }
  s = P->ex.make_add(P->add, outs, G.add_src, insts, G.add_mult);
  if (s != PES_OK) return s;

  if (P->with_vjp) {
    std::vector<pes::ConvJob> fwdm(G.vjp_jobs.begin(), G.vjp_jobs.begin() + G.vjp_fwd_jobs);
    std::vector<pes::ConvJob> corr(G.vjp_jobs.begin() + G.vjp_fwd_jobs, G.vjp_jobs.end());
    std::vector<pes::ConvJob> monly = G.vjp_mjobs;
    resolve_local_deps(monly);  // M_m * F_m (monomials with powers) waits for M_m
    s = P->ex.make_joblist(P->vjp_fwd, fwdm);
    if (s == PES_OK) s = P->ex.make_joblist(P->vjp_m, monly);
    if (s == PES_OK) s = P->ex.make_joblist(P->vjp_corr, corr);
    if (s != PES_OK) return s;
    std::vector<pes::AddOut> gouts;
    std::vector<pes::CopyRow> urow, un;
    if (complex_series) {
      // VJP slot s of the real layout holds its parts in 2s and 2s + 1;
      // upstream, grad_coeff and grad_input are real block then imaginary block
      for (int32_t i = 0; i < n; ++i)
        for (int part = 0; part < 2; ++part) {
          const size_t o = static_cast<size_t>(2 * (1 + i) + part);
          gouts.push_back({static_cast<int64_t>(2 * (G.slot_g0 + i) + part), 0, 0, 0, G.add_ptr[o], G.add_ptr[o + 1]});
        }
      const int64_t uim = static_cast<int64_t>(k) * D1;
      urow.push_back({0, D1, 2, 0, 2 * G.slot_u, 0});
      urow.push_back({uim, D1, 2, 0, 2 * G.slot_u + 1, 0});
      for (int part = 0; part < 2; ++part) {
        const int64_t co = part ? cim : 0, io = part ? iim : 0;
        un.push_back({co, (N + 1) * D1, 0, 0, 2 * G.slot_u + part, 0});
        for (int32_t m = 1; m <= N; ++m)
          un.push_back({co + m * D1, (N + 1) * D1, 0, 0, 2 * (G.slot_r0 + m - 1) + part, 0});
        for (int32_t i = 0; i < n; ++i) un.push_back({io + i * D1, n * D1, 1, 0, 2 * (G.slot_r0 + N + i) + part, 0});
      }
    } else if (np == 0) {
      // gradient series into workspace slots (digit form)
      for (int32_t i = 0; i < n; ++i)
        gouts.push_back({static_cast<int64_t>(G.slot_g0 + i), 0, 0, 0, G.add_ptr[1 + i], G.add_ptr[2 + i]});
      urow.push_back({0, D1, 2, 0, G.slot_u, 0});
      // unpack: grad_coeff (buffer 0) <- u, r_m ; grad_input (buffer 1) <- r_{N+i}
      un.push_back({0, (N + 1) * D1, 0, 0, G.slot_u, 0});
      for (int32_t m = 1; m <= N; ++m) un.push_back({m * D1, (N + 1) * D1, 0, 0, G.slot_r0 + m - 1, 0});
      for (int32_t i = 0; i < n; ++i) un.push_back({i * D1, n * D1, 1, 0, G.slot_r0 + N + i, 0});
    } else {
      // system: the nonempty Jacobian series into workspace slots; upstream
      // [k][P][d+1]; grad_coeff rows as the coefficient buffer (constant of p
      // <- u_p, monomial m <- r_m); grad_input[i] = sum_p of the correlations
      // of u_p with the Jacobian series (p, i), summed exactly and rounded once
      const int64_t cl = static_cast<int64_t>(N + np) * D1;
      std::vector<pes::AddOut> giouts;
      std::vector<int32_t> gicontrib;
      for (int32_t p = 0; p < np; ++p) {
        urow.push_back({p * D1, np * D1, 2, 0, G.slot_up0 + p, 0});
        const int32_t m0 = (*poly_ptr)[static_cast<size_t>(p)], m1 = (*poly_ptr)[static_cast<size_t>(p) + 1];
        un.push_back({static_cast<int64_t>(m0 + p) * D1, cl, 0, 0, G.slot_up0 + p, 0});
        for (int32_t m = m0; m < m1; ++m)
          un.push_back({static_cast<int64_t>(m + p + 1) * D1, cl, 0, 0, G.slot_r0 + m, 0});
        for (int32_t i = 0; i < n; ++i) {
          const size_t o = static_cast<size_t>(np + p * n + i);
          if (G.add_ptr[o + 1] > G.add_ptr[o])
            gouts.push_back({static_cast<int64_t>(G.slot_J0 + p * n + i), 0, 0, 0, G.add_ptr[o], G.add_ptr[o + 1]});
        }
      }
      for (int32_t i = 0; i < n; ++i) {
        const int32_t c0 = static_cast<int32_t>(gicontrib.size());
        for (int32_t p = 0; p < np; ++p) {
          const size_t o = static_cast<size_t>(np + p * n + i);
          if (G.add_ptr[o + 1] > G.add_ptr[o]) gicontrib.push_back(G.slot_rJ0 + p * n + i);
        }
        giouts.push_back({i * D1, n * D1, 0, 0, c0, static_cast<int32_t>(gicontrib.size())});
      }
      s = P->ex.make_add(P->add_gi, giouts, gicontrib, insts);
      if (s != PES_OK) return s;
    }
    s = P->ex.make_add(P->add_g, gouts, G.add_src, insts, G.add_mult);
    if (s != PES_OK) return s;
    P->pack_u.n = static_cast<int32_t>(urow.size());
    s = P->ex.put(&P->pack_u.rows, urow);
    if (s != PES_OK) return s;
    P->unpack.n = static_cast<int32_t>(un.size());
    s = P->ex.put(&P->unpack.rows, un);
    if (s != PES_OK) return s;
  }
  *out = P.release();
  return PES_OK;
}
}  // namespace

extern "C" void pes_plan_destroy(pes_plan_t plan) { delete plan; }

// First call of a plan built with `autotune`: tune its convolution launch by
// running `run` (the call's own work on the caller's buffers), then give the
// VJP job lists the same launch shape.
template <class Run>
static pes_status tune_plan(pes_plan_t plan, Run run, cudaStream_t st) {
  if (!plan->autotune || plan->tuned) return PES_OK;
  plan->tuned = true;
  Exec& E = plan->ex;
  pes_status ts = tune_launch(E, plan->fwd, tune_key(E, plan->fwd.n, plan->signature), run, st);
  if (ts != PES_OK) return ts;
  plan->vjp_fwd.grid = plan->vjp_m.grid = plan->vjp_corr.grid = 0;
  for (JobList* L : {&plan->vjp_fwd, &plan->vjp_m, &plan->vjp_corr}) {
    if (L->n == 0) continue;
    ts = E.configure(E.threads, E.blocks_per_sm, E.depth, E.split, *L);
    if (ts != PES_OK) return ts;
  }
  return PES_OK;
}

extern "C" pes_status pes_eval_grad(pes_plan_t plan, const double* coeff, const double* input, double* value,
                                    double* grad, void* stream) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  if (!coeff || !input || !value || !grad) return fail(PES_EINVAL, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Exec& E = plan->ex;
  {
    auto run = [&](cudaStream_t s2) -> pes_status {
      PES_CUDA(pes::launch_prologue(E.ctrl, s2));
      PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, s2));
      PES_CUDA(E.run_dag(plan->fwd, 0, s2));
      PES_CUDA(E.run_add(plan->add, value, grad, s2));
      return PES_OK;
    };
    pes_status ts = tune_plan(plan, run, st);
    if (ts != PES_OK) return ts;
  }
  PES_CUDA(E.mark(0, st));
  PES_CUDA(pes::launch_prologue(E.ctrl, st));
  PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, st));
  PES_CUDA(E.mark(1, st));
  PES_CUDA(E.run_dag(plan->fwd, 0, st));
  PES_CUDA(E.mark(2, st));
  PES_CUDA(E.run_add(plan->add, value, grad, st));
  PES_CUDA(E.mark(3, st));
  PES_CUDA(E.mark(4, st));
  E.last_launches = 1 + Exec::launches(plan->pack) + Exec::launches(plan->fwd) + Exec::launches(plan->add);
  return PES_OK;
}

// ---- one polynomial split over ranks (Sec. 5: monomials are independent up to
// the addition jobs; the exchange is exact integer arithmetic) ----------------

extern "C" pes_status pes_shard_range(const int32_t* supp_ptr, int32_t N, int32_t world, int32_t rank,
                                      int32_t* m_begin, int32_t* m_end) {
  if (N < 0 || world < 1 || rank < 0 || rank >= world || !m_begin || !m_end || (N > 0 && !supp_ptr))
    return fail(PES_EINVAL, "bad sizes, rank or NULL pointer");
  // cost of monomial m: its convolution jobs, 3 n_m - 3 (one for n_m = 1)
  std::vector<int64_t> pre(static_cast<size_t>(N) + 1, 0);
  for (int32_t m = 0; m < N; ++m) {
    const int64_t nm = supp_ptr[m + 1] - supp_ptr[m];
    if (nm < 1) return fail(PES_EINVAL, "empty monomial " + std::to_string(m));
    pre[static_cast<size_t>(m) + 1] = pre[static_cast<size_t>(m)] + (nm >= 2 ? 3 * nm - 3 : 1);
  }
  const int64_t W = pre.back();
  // rank r takes the monomials whose cost prefix starts in [r W / world, (r+1) W / world)
  auto bound = [&](int32_t r) -> int32_t {
    if (r <= 0) return 0;
    if (r >= world) return N;
    int32_t m = 0;
    while (m < N && pre[static_cast<size_t>(m)] * world < static_cast<int64_t>(r) * W) ++m;
    return m;
  };
  *m_begin = bound(rank);
  *m_end = bound(rank + 1);
  return PES_OK;
}

namespace {
pes_status check_shardable(pes_plan_t plan) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  if (plan->complex_series || plan->prog.system_P > 0)
    return fail(PES_EINVAL, "partial sums take real single-polynomial plans (not complex, not systems)");
  return PES_OK;
}
}  // namespace

extern "C" pes_status pes_partial_grids(pes_plan_t plan, const double* coeff, const double* input, int32_t* grids,
                                        void* stream) {
  pes_status s = check_shardable(plan);
  if (s != PES_OK) return s;
  if (!coeff || !input || !grids) return fail(PES_EINVAL, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Exec& E = plan->ex;
  auto run = [&](cudaStream_t s2) -> pes_status {
    PES_CUDA(pes::launch_prologue(E.ctrl, s2));
    PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, s2));
    PES_CUDA(E.run_dag(plan->fwd, 0, s2));
    PES_CUDA(E.run_add(plan->add, nullptr, nullptr, s2, 1, grids, nullptr));
    return PES_OK;
  };
  s = tune_plan(plan, run, st);
  if (s != PES_OK) return s;
  s = run(st);
  if (s != PES_OK) return s;
  E.last_launches = 1 + Exec::launches(plan->pack) + Exec::launches(plan->fwd) + Exec::launches(plan->add);
  return PES_OK;
}

extern "C" pes_status pes_partial_sums(pes_plan_t plan, const int32_t* grids, int64_t* acc, void* stream) {
  pes_status s = check_shardable(plan);
  if (s != PES_OK) return s;
  if (!grids || !acc) return fail(PES_EINVAL, "NULL buffer");
  Exec& E = plan->ex;
  PES_CUDA(E.run_add(plan->add, nullptr, nullptr, static_cast<cudaStream_t>(stream), 2, const_cast<int32_t*>(grids),
                     reinterpret_cast<long long*>(acc)));
  E.last_launches = Exec::launches(plan->add);
  return PES_OK;
}

extern "C" pes_status pes_round_sums(pes_plan_t plan, const int32_t* grids, const int64_t* acc, double* value,
                                     double* grad, void* stream) {
  pes_status s = check_shardable(plan);
  if (s != PES_OK) return s;
  if (!grids || !acc || !value || !grad) return fail(PES_EINVAL, "NULL buffer");
  pes::RoundArgs a{grids, reinterpret_cast<const long long*>(acc), value, grad, plan->prog.n, plan->prog.d};
  PES_CUDA(pes::launch_round_sums(a, plan->ex.k, plan->ex.arith, static_cast<cudaStream_t>(stream)));
  return PES_OK;
}

extern "C" pes_status pes_round_sums_host(int32_t k, int32_t arith, int32_t n, int32_t d, const int32_t* grids,
                                          const int64_t* acc, double* value, double* grad) {
  if (!valid_k(k)) return fail(PES_EUNSUPPORTED_K, "k must be one of 1,2,3,4,5,8,10");
  if (arith != pes::ARITH_INT && arith != pes::ARITH_FP64) return fail(PES_EINVAL, "arith must be 0 or 1");
  if (n < 1 || d < 0 || d > pes::kMaxDegree || !grids || !acc || !value || !grad)
    return fail(PES_EINVAL, "bad sizes or NULL buffer");
  pes::RoundArgs a{grids, reinterpret_cast<const long long*>(acc), value, grad, n, d};
  return pes::round_sums_host(k, arith, a) == 0 ? PES_OK : fail(PES_EINTERNAL, "rounding");
}

extern "C" pes_status pes_eval_system(pes_plan_t plan, const double* coeff, const double* input, double* value,
                                      double* jac, int32_t layout, void* stream) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  if (plan->prog.system_P == 0) return fail(PES_EINVAL, "plan is not a system (pes_plan_system)");
  if (layout != PES_LAYOUT_SERIES && layout != PES_LAYOUT_MATRIX) return fail(PES_EINVAL, "unknown layout");
  if (layout == PES_LAYOUT_SERIES) return pes_eval_grad(plan, coeff, input, value, jac, stream);
  if (!coeff || !input || !value || !jac) return fail(PES_EINVAL, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Exec& E = plan->ex;
  {
    // both layouts share the job list and its launch shape
    auto run = [&](cudaStream_t s2) -> pes_status {
      PES_CUDA(pes::launch_prologue(E.ctrl, s2));
      PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, s2));
      PES_CUDA(E.run_dag(plan->fwd, 0, s2));
      PES_CUDA(E.run_add(plan->add_mat, value, jac, s2));
      return PES_OK;
    };
    pes_status ts = tune_plan(plan, run, st);
    if (ts != PES_OK) return ts;
  }
  PES_CUDA(E.mark(0, st));
  PES_CUDA(pes::launch_prologue(E.ctrl, st));
  PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, st));
  PES_CUDA(E.mark(1, st));
  PES_CUDA(E.run_dag(plan->fwd, 0, st));
  PES_CUDA(E.mark(2, st));
  PES_CUDA(E.run_add(plan->add_mat, value, jac, st));
  PES_CUDA(E.mark(3, st));
  PES_CUDA(E.mark(4, st));
  E.last_launches = 1 + Exec::launches(plan->pack) + Exec::launches(plan->fwd) + Exec::launches(plan->add_mat);
  return PES_OK;
}

extern "C" pes_status pes_vjp(pes_plan_t plan, const double* coeff, const double* input, const double* upstream,
                              double* grad_input, double* grad_coeff, int32_t reuse_forward, void* stream) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  if (!plan->with_vjp) return fail(PES_EINVAL, "plan was built without with_vjp");
  if (!upstream || !grad_input || !grad_coeff || (!reuse_forward && (!coeff || !input)))
    return fail(PES_EINVAL, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Exec& E = plan->ex;
  PES_CUDA(E.mark(0, st));
  PES_CUDA(pes::launch_prologue(E.ctrl, st));
  if (reuse_forward) {
    PES_CUDA(E.run_pack(plan->pack_u, nullptr, nullptr, upstream, st));
    PES_CUDA(E.mark(1, st));
    PES_CUDA(E.run_dag(plan->vjp_m, 0, st));
    E.last_launches = 1 + Exec::launches(plan->pack_u) + Exec::launches(plan->vjp_m);
  } else {
    PES_CUDA(E.run_pack(plan->pack, coeff, input, nullptr, st));
    PES_CUDA(E.run_pack(plan->pack_u, nullptr, nullptr, upstream, st));
    PES_CUDA(E.mark(1, st));
    PES_CUDA(E.run_dag(plan->vjp_fwd, 0, st));
    E.last_launches = 1 + Exec::launches(plan->pack) + Exec::launches(plan->pack_u) + Exec::launches(plan->vjp_fwd);
  }
  E.last_launches += Exec::launches(plan->add_g) + Exec::launches(plan->vjp_corr) + Exec::launches(plan->unpack);
  PES_CUDA(E.run_add(plan->add_g, nullptr, nullptr, st));
  PES_CUDA(E.run_dag(plan->vjp_corr, 1, st));
  PES_CUDA(E.mark(2, st));
  if (plan->prog.system_P > 0) {
    PES_CUDA(E.run_add(plan->add_gi, grad_input, nullptr, st));  // sum over the polynomials
    E.last_launches += Exec::launches(plan->add_gi);
  }
  PES_CUDA(E.mark(3, st));
  PES_CUDA(E.run_unpack(plan->unpack, grad_coeff, grad_input, st));
  PES_CUDA(E.mark(4, st));
  return PES_OK;
}

extern "C" pes_status pes_workspace_io(pes_plan_t plan, void* buffer, int32_t to_buffer, void* stream) {
  if (!plan || !buffer) return fail(PES_EINVAL, "NULL argument");
  const size_t bytes = plan->ex.ws_words * sizeof(int32_t);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (to_buffer)
    PES_CUDA(cudaMemcpyAsync(buffer, plan->ex.ws, bytes, cudaMemcpyDeviceToDevice, st));
  else
    PES_CUDA(cudaMemcpyAsync(plan->ex.ws, buffer, bytes, cudaMemcpyDeviceToDevice, st));
  return PES_OK;
}

extern "C" pes_status pes_last_timing(pes_plan_t plan, double* ms, int32_t* launches) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  return plan->ex.last_timing(ms, launches);
}

extern "C" pes_status pes_check(pes_plan_t plan, void* stream) {
  if (!plan) return fail(PES_EINVAL, "plan is NULL");
  return plan->ex.check(static_cast<cudaStream_t>(stream));
}

extern "C" pes_status pes_get_plan_info(pes_plan_t plan, pes_plan_info* info) {
  if (!plan || !info) return fail(PES_EINVAL, "NULL argument");
  const pes::Program1& G = plan->prog;
  std::memset(info, 0, sizeof(*info));
  info->conv_jobs = static_cast<int64_t>(G.jobs.size());
  info->layers = G.n_layers;
  info->add_terms = static_cast<int64_t>(G.add_src.size());
  int64_t nonempty = 0;
  for (size_t o = 0; o + 1 < G.add_ptr.size(); ++o) nonempty += G.add_ptr[o + 1] > G.add_ptr[o];
  info->add_jobs = info->add_terms - nonempty;
  info->workspace_bytes = plan->ws_bytes;
  info->vjp_conv_jobs = plan->with_vjp ? G.vjp_fwd_jobs - static_cast<int64_t>(G.jobs.size()) : 0;
  info->vjp_corr_jobs = plan->with_vjp ? static_cast<int64_t>(G.vjp_jobs.size()) - G.vjp_fwd_jobs : 0;
  info->digits = pes::digits_of_k(plan->ex.k, plan->ex.arith);
  info->grid = plan->fwd.grid;
  info->threads = plan->ex.threads;
  info->smem_bytes = static_cast<int32_t>(plan->ex.smem);
  info->arith = plan->ex.arith;
  info->staging = plan->ex.depth;
  info->split = plan->ex.split;
  info->complex_series = plan->complex_series ? 1 : 0;
  info->system_P = plan->prog.system_P;
  info->tile = plan->ex.tile;
  return PES_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
//
// Instances are grouped by the CTA shape their degree needs (integer pipe: one
// lane per output coefficient, d+1 rounded up to whole warps; FP64 pipe: 128
// threads).  Every group is one persistent launch over its instances'
// concatenated job tables (sorted by layer, larger degree first); the groups run
// on forked streams inside one captured CUDA graph.

namespace {

struct Group {
  Exec ex;
  JobList fwd;
  AddTable add;
  CopyTable pack;
  std::vector<int32_t> members;
  int64_t conv_jobs = 0, terms = 0;
  uint64_t signature = 1469598103934665603ull;  // FNV-1a over the job structure
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  ~Group() {
    if (done) cudaEventDestroy(done);
    if (stream) cudaStreamDestroy(stream);
  }
};

}  // namespace

struct pes_batch_s {
  std::vector<std::unique_ptr<Group>> groups;
  int32_t count = 0, k = 0;
  bool autotune = false, tuned = false, profile = false;
  std::vector<int64_t> coeff_off, input_off, value_off, grad_off;
  int64_t conv_jobs = 0, layers = 0, add_terms = 0, add_jobs = 0;
  // CUDA graph of one call, re-instantiated when the caller's buffers change
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int32_t last_launches = 0;
  ~pes_batch_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    groups.clear();
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

extern "C" pes_status pes_plan_batch(int32_t count, const int32_t* n, const int32_t* N, const int32_t* d,
                                     const int32_t* supp_ptr, const int32_t* supp_idx, int32_t k,
                                     const pes_options* opt, pes_batch_t* out) {
  return pes_plan_batch_powers(count, n, N, d, supp_ptr, supp_idx, nullptr, k, opt, out);
}

extern "C" pes_status pes_plan_batch_powers(int32_t count, const int32_t* n, const int32_t* N, const int32_t* d,
                                            const int32_t* supp_ptr, const int32_t* supp_idx,
                                            const int32_t* supp_exp, int32_t k, const pes_options* opt,
                                            pes_batch_t* out) {
  if (!out) return fail(PES_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !n || !N || !d || !supp_ptr) return fail(PES_EINVAL, "bad batch arguments");
  if (!valid_k(k)) return fail(PES_EUNSUPPORTED_K, "k must be one of 1,2,3,4,5,8,10");
  pes_options o;
  pes_status s = parse_options(opt, o);
  if (s != PES_OK) return s;
  std::unique_ptr<pes_batch_s> B(new (std::nothrow) pes_batch_s());
  if (!B) return fail(PES_ENOMEM, "batch");
  B->count = count;
  B->k = k;
  B->autotune = o.autotune != 0;
  B->profile = o.profile != 0;

  std::vector<pes::Program1> progs(static_cast<size_t>(count));
  B->coeff_off.assign(static_cast<size_t>(count) + 1, 0);
  B->input_off.assign(static_cast<size_t>(count) + 1, 0);
  B->value_off.assign(static_cast<size_t>(count) + 1, 0);
  B->grad_off.assign(static_cast<size_t>(count) + 1, 0);
  // (arith, threads, tiled) -> instances; the tiled kernel takes the degrees
  // whose whole series do not fit in shared memory
  std::map<std::tuple<int32_t, int32_t, int32_t>, std::vector<int32_t>> classes;
  const int optin = device_optin();
  int64_t prow = 0, qidx = 0;
  for (int32_t b = 0; b < count; ++b) {
    if (d[b] < 0 || d[b] > pes::kMaxDegree) return fail(PES_EINVAL, "instance " + std::to_string(b) + ": bad degree");
    pes::Supports sup;
    const int32_t* bp = supp_ptr + prow;
    const int32_t* bi = supp_idx ? supp_idx + qidx : nullptr;
    const int32_t* be = supp_exp ? supp_exp + qidx : nullptr;
    s = build_supports(bp, bi, N[b], n[b], sup, be);
    if (s != PES_OK) return fail(s, "instance " + std::to_string(b) + ": " + g_last_error);
    progs[static_cast<size_t>(b)] = pes::compile(sup, d[b], false, false);
    const int64_t D1 = d[b] + 1;
    B->coeff_off[static_cast<size_t>(b) + 1] = B->coeff_off[static_cast<size_t>(b)] + k * (N[b] + 1) * D1;
    B->input_off[static_cast<size_t>(b) + 1] = B->input_off[static_cast<size_t>(b)] + k * n[b] * D1;
    B->value_off[static_cast<size_t>(b) + 1] = B->value_off[static_cast<size_t>(b)] + k * D1;
    B->grad_off[static_cast<size_t>(b) + 1] = B->grad_off[static_cast<size_t>(b)] + k * n[b] * D1;
    prow += N[b] + 1;
    qidx += sup.ptr.back();
    const int32_t ar = resolve_arith(k, o.arith, d[b]);
    const bool tiled = o.tile > 0 || !whole_series_fits(k, ar, d[b], o.threads, optin);
    // default CTA: one lane per coefficient within the cap
    const int32_t T = std::min((2 * ((d[b] + 2) / 2) + 31) / 32 * 32, pes::dag_max_threads(k));
    classes[std::make_tuple(ar, ar == pes::ARITH_INT && !tiled ? T : 0, tiled ? 1 : 0)].push_back(b);
  }

  for (auto& cls : classes) {
    std::unique_ptr<Group> G(new (std::nothrow) Group());
    if (!G) return fail(PES_ENOMEM, "batch group");
    G->members = cls.second;
    const size_t ng = G->members.size();
    std::vector<pes::InstInfo> insts(ng);
    int64_t wsbase = 0;
    for (size_t u = 0; u < ng; ++u) {
      const int32_t b = G->members[u];
      const int32_t S = pes::series_stride(d[b]);
      const int64_t slots = progs[static_cast<size_t>(b)].n_slots;
      const int64_t sstride = pes::ws_slot_words(k, std::get<0>(cls.first), S);
      insts[u] = pes::InstInfo{wsbase, sstride, S, d[b]};
      wsbase += slots * sstride;
    }
    pes_options og = o;
    og.arith = std::get<0>(cls.first);
    og.threads = std::max(o.threads, std::get<1>(cls.first));
    if (std::get<2>(cls.first)) og.tile = o.tile > 0 ? o.tile : pes::kDefaultTile;
    s = G->ex.init(k, og, insts, static_cast<size_t>(wsbase));
    if (s != PES_OK) return s;

    struct Ref {
      int32_t layer, d, inst, local;
    };
    std::vector<Ref> refs;
    for (size_t u = 0; u < ng; ++u) {
      const int32_t b = G->members[u];
      for (size_t t = 0; t < progs[static_cast<size_t>(b)].jobs.size(); ++t)
        refs.push_back({progs[static_cast<size_t>(b)].jobs[t].layer, d[b], static_cast<int32_t>(u),
                        static_cast<int32_t>(t)});
    }
    std::stable_sort(refs.begin(), refs.end(), [](const Ref& x, const Ref& y) {
      if (x.layer != y.layer) return x.layer < y.layer;
      return x.d > y.d;
    });
    std::vector<std::vector<int32_t>> gidx(ng);
    for (size_t u = 0; u < ng; ++u) gidx[u].assign(progs[static_cast<size_t>(G->members[u])].jobs.size(), -1);
    for (size_t g = 0; g < refs.size(); ++g)
      gidx[static_cast<size_t>(refs[g].inst)][static_cast<size_t>(refs[g].local)] = static_cast<int32_t>(g);
    std::vector<pes::ConvJob> jobs(refs.size());
    for (size_t g = 0; g < refs.size(); ++g) {
      const auto& gi = gidx[static_cast<size_t>(refs[g].inst)];
      pes::ConvJob j = progs[static_cast<size_t>(G->members[static_cast<size_t>(refs[g].inst)])]
                           .jobs[static_cast<size_t>(refs[g].local)];
      j.dep1 = j.dep1 >= 0 ? gi[static_cast<size_t>(j.dep1)] : -1;
      j.dep2 = j.dep2 >= 0 ? gi[static_cast<size_t>(j.dep2)] : -1;
      j.inst = refs[g].inst;
      jobs[g] = j;
      B->layers = std::max<int64_t>(B->layers, j.layer);
      fnv_mix(G->signature, j.layer);
      fnv_mix(G->signature, refs[g].d);
      G->terms += static_cast<int64_t>(refs[g].d + 1) * (refs[g].d + 2) / 2;
    }
    G->conv_jobs = static_cast<int64_t>(jobs.size());
    B->conv_jobs += G->conv_jobs;
    G->ex.choose_split(jobs);
    s = G->ex.make_joblist(G->fwd, jobs);
    if (s != PES_OK) return s;

    std::vector<pes::CopyRow> rows;
    std::vector<pes::AddOut> outs;
    std::vector<int32_t> contrib, mult;
    for (size_t u = 0; u < ng; ++u) {
      const int32_t b = G->members[u];
      const int32_t iu = static_cast<int32_t>(u);
      const pes::Program1& P = progs[static_cast<size_t>(b)];
      const int64_t D1 = d[b] + 1;
      const int64_t co = B->coeff_off[static_cast<size_t>(b)], io = B->input_off[static_cast<size_t>(b)];
      for (int32_t m = 0; m <= N[b]; ++m) rows.push_back({co + m * D1, (N[b] + 1) * D1, 0, iu, m, 0});
      for (int32_t i = 0; i < n[b]; ++i) rows.push_back({io + i * D1, n[b] * D1, 1, iu, 1 + N[b] + i, 0});
      const int32_t c0 = static_cast<int32_t>(contrib.size());
      contrib.insert(contrib.end(), P.add_src.begin(), P.add_src.end());
      mult.insert(mult.end(), P.add_mult.begin(), P.add_mult.end());
      outs.push_back({B->value_off[static_cast<size_t>(b)], D1, 0, iu, c0 + P.add_ptr[0], c0 + P.add_ptr[1]});
      for (int32_t i = 0; i < n[b]; ++i)
        outs.push_back({B->grad_off[static_cast<size_t>(b)] + i * D1, n[b] * D1, 1, iu, c0 + P.add_ptr[1 + i],
                        c0 + P.add_ptr[2 + i]});
      B->add_terms += static_cast<int64_t>(P.add_src.size());
      for (size_t oo = 0; oo + 1 < P.add_ptr.size(); ++oo)
        B->add_jobs += std::max(0, P.add_ptr[oo + 1] - P.add_ptr[oo] - 1);
    }
    G->pack.n = static_cast<int32_t>(rows.size());
    s = G->ex.put(&G->pack.rows, rows);
    if (s == PES_OK) s = G->ex.make_add(G->add, outs, contrib, insts, mult);
    if (s != PES_OK) return s;
    PES_CUDA(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
    PES_CUDA(cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming));
    B->groups.push_back(std::move(G));
  }
  PES_CUDA(cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
  PES_CUDA(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
  if (B->profile)
    for (cudaEvent_t& e : B->ev) PES_CUDA(cudaEventCreate(&e));
  *out = B.release();
  return PES_OK;
}

extern "C" void pes_batch_destroy(pes_batch_t batch) { delete batch; }

extern "C" pes_status pes_batch_offsets(pes_batch_t batch, int64_t* coeff_off, int64_t* input_off,
                                        int64_t* value_off, int64_t* grad_off) {
  if (!batch) return fail(PES_EINVAL, "batch is NULL");
  const size_t n = batch->coeff_off.size();
  if (coeff_off) std::memcpy(coeff_off, batch->coeff_off.data(), n * sizeof(int64_t));
  if (input_off) std::memcpy(input_off, batch->input_off.data(), n * sizeof(int64_t));
  if (value_off) std::memcpy(value_off, batch->value_off.data(), n * sizeof(int64_t));
  if (grad_off) std::memcpy(grad_off, batch->grad_off.data(), n * sizeof(int64_t));
  return PES_OK;
}

static pes_status group_record(Group& G, const double* coeff, const double* input, double* value, double* grad,
                               cudaStream_t st) {
  Exec& E = G.ex;
  PES_CUDA(pes::launch_prologue(E.ctrl, st));
  PES_CUDA(E.run_pack(G.pack, coeff, input, nullptr, st));
  PES_CUDA(E.run_dag(G.fwd, 0, st));
  PES_CUDA(E.run_add(G.add, value, grad, st));
  return PES_OK;
}

static pes_status batch_record(pes_batch_t B, const double* coeff, const double* input, double* value,
                               double* grad, cudaStream_t st) {
  if (B->groups.size() == 1) return group_record(*B->groups[0], coeff, input, value, grad, st);
  PES_CUDA(cudaEventRecord(B->fork, st));
  for (auto& G : B->groups) {
    PES_CUDA(cudaStreamWaitEvent(G->stream, B->fork, 0));
    pes_status s = group_record(*G, coeff, input, value, grad, G->stream);
    if (s != PES_OK) return s;
    PES_CUDA(cudaEventRecord(G->done, G->stream));
  }
  for (auto& G : B->groups) PES_CUDA(cudaStreamWaitEvent(st, G->done, 0));
  return PES_OK;
}

// Pick the launch shape of every group by timing its launches on the caller's
// data (see tune_launch).
static pes_status batch_autotune(pes_batch_t B, const double* coeff, const double* input, double* value,
                                 double* grad, cudaStream_t st) {
  for (auto& Gp : B->groups) {
    Group& G = *Gp;
    auto run = [&](cudaStream_t s2) { return group_record(G, coeff, input, value, grad, s2); };
    pes_status s = tune_launch(G.ex, G.fwd, tune_key(G.ex, G.conv_jobs, G.signature), run, st);
    if (s != PES_OK) return s;
  }
  return PES_OK;
}

extern "C" pes_status pes_eval_grad_batch(pes_batch_t batch, const double* coeff, const double* input, double* value,
                                          double* grad, void* stream) {
  if (!batch) return fail(PES_EINVAL, "batch is NULL");
  if (!coeff || !input || !value || !grad) return fail(PES_EINVAL, "NULL buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (batch->autotune && !batch->tuned) {
    pes_status s = batch_autotune(batch, coeff, input, value, grad, st);
    if (s != PES_OK) return s;
    batch->tuned = true;
  }
  const void* key[4] = {coeff, input, value, grad};
  if (!batch->gexec || std::memcmp(key, batch->gkey, sizeof(key)) != 0) {
    if (batch->gexec) {
      cudaGraphExecDestroy(batch->gexec);
      batch->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    PES_CUDA(cudaStreamBeginCapture(batch->capture_stream, cudaStreamCaptureModeThreadLocal));
    pes_status s = batch_record(batch, coeff, input, value, grad, batch->capture_stream);
    cudaError_t e = cudaStreamEndCapture(batch->capture_stream, &graph);
    if (s != PES_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&batch->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    std::memcpy(batch->gkey, key, sizeof(key));
  }
  if (batch->profile) PES_CUDA(cudaEventRecord(batch->ev[0], st));
  PES_CUDA(cudaGraphLaunch(batch->gexec, st));
  if (batch->profile) PES_CUDA(cudaEventRecord(batch->ev[1], st));
  batch->last_launches = 0;
  for (auto& G : batch->groups)
    batch->last_launches += 1 + Exec::launches(G->pack) + Exec::launches(G->fwd) + Exec::launches(G->add);
  return PES_OK;
}

extern "C" pes_status pes_batch_last_timing(pes_batch_t batch, double* ms, int32_t* launches) {
  if (!batch) return fail(PES_EINVAL, "batch is NULL");
  if (!batch->profile) return fail(PES_EINVAL, "built without profile = 1");
  PES_CUDA(cudaEventSynchronize(batch->ev[1]));
  float t = 0.f;
  PES_CUDA(cudaEventElapsedTime(&t, batch->ev[0], batch->ev[1]));
  if (ms) {
    ms[0] = 0.0;
    ms[1] = t;  // the whole graph (pack, convolutions and additions of every group)
    ms[2] = 0.0;
    ms[3] = 0.0;
  }
  if (launches) *launches = batch->last_launches;
  return PES_OK;
}

extern "C" pes_status pes_batch_check(pes_batch_t batch, void* stream) {
  if (!batch) return fail(PES_EINVAL, "batch is NULL");
  PES_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  for (auto& G : batch->groups) {
    pes_status s = G->ex.check(G->stream);
    if (s != PES_OK) return s;
  }
  return PES_OK;
}

extern "C" pes_status pes_get_batch_info(pes_batch_t batch, pes_plan_info* info) {
  if (!batch || !info) return fail(PES_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->conv_jobs = batch->conv_jobs;
  info->layers = batch->layers;
  info->add_terms = batch->add_terms;
  info->add_jobs = batch->add_jobs;
  size_t ws = 0;
  for (auto& G : batch->groups) ws += G->ex.ws_words * sizeof(int32_t);
  info->workspace_bytes = static_cast<int64_t>(ws);
  const Exec& E0 = batch->groups.front()->ex;
  info->digits = pes::digits_of_k(batch->k, E0.arith);
  info->grid = static_cast<int32_t>(batch->groups.size());  // number of groups (persistent launches)
  info->threads = E0.threads;
  info->smem_bytes = static_cast<int32_t>(E0.smem);
  info->arith = E0.arith;
  info->staging = E0.depth;
  info->split = E0.split;
  for (auto& G : batch->groups) info->tile = std::max(info->tile, G->ex.tile);  // tiled groups, if any
  return PES_OK;
}

// ---------------------------------------------------------------------------
// multiple double numbers, costs, FP64 peak
// ---------------------------------------------------------------------------

extern "C" pes_status pes_md_binary(int32_t op, int32_t k, const double* x, const double* y, double* out,
                                    int64_t count, void* stream) {
  if (!valid_k(k)) return fail(PES_EUNSUPPORTED_K, "k must be one of 1,2,3,4,5,8,10");
  if (op != 0 && op != 1) return fail(PES_EINVAL, "op must be 0 (add) or 1 (mul)");
  if (count < 0 || (count > 0 && (!x || !y || !out))) return fail(PES_EINVAL, "bad buffers");
  PES_CUDA(pes::launch_md_binary(op, k, x, y, out, count, static_cast<cudaStream_t>(stream)));
  return PES_OK;
}

extern "C" pes_status pes_md_costs(int32_t k, double* mul_ops, double* add_ops) {
  if (!valid_k(k)) return fail(PES_EUNSUPPORTED_K, "k must be one of 1,2,3,4,5,8,10");
  double mul, add;
  if (k == 10) {
    mul = 3089.0;  // Sec. 6.2: 952 additions, 1743 subtractions, 394 multiplications
    add = 397.0;   // Sec. 6.2: 139 additions, 258 subtractions
  } else if (k == 1) {
    mul = 1.0;
    add = 1.0;
  } else {
    // FP64 operations of md.cuh: md_mul = TwoProd (2) for orders <= k-2, each
    // deposit at order s costs 6 (k - s) + 1, then renorm<k+1,k> (9 k);
    // md_add = renorm<2k,k> (9 (2k - 1)).
    double m = 0.0;
    for (int s = 0; s < k; ++s)
      for (int p = 0; p <= s; ++p) {
        if (s < k - 1)
          m += 2.0 + (6.0 * (k - s) + 1.0) + (6.0 * (k - s - 1) + 1.0);
        else
          m += 1.0 + (6.0 * (k - s) + 1.0);
      }
    mul = m + 9.0 * k;
    add = 9.0 * (2 * k - 1);
  }
  if (mul_ops) *mul_ops = mul;
  if (add_ops) *add_ops = add;
  return PES_OK;
}

extern "C" pes_status pes_fp64_peak(int32_t repeats, double* tflops) {
  if (!tflops) return fail(PES_EINVAL, "tflops is NULL");
  int dev = 0, nsm = 0;
  PES_CUDA(cudaGetDevice(&dev));
  PES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  const int threads = 256, blocks = nsm * 4, iters = 4096;
  PES_CUDA(cudaMalloc(&sink, sizeof(double) * static_cast<size_t>(blocks)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  pes::launch_fp64_peak(sink, blocks, threads, iters / 8, nullptr);  // warm-up
  for (int r = 0; r < std::max(1, repeats); ++r) {
    cudaEventRecord(e0, nullptr);
    pes::launch_fp64_peak(sink, blocks, threads, iters, nullptr);
    cudaEventRecord(e1, nullptr);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 peak kernel");
  const double fmas = static_cast<double>(blocks) * threads * iters * 8.0;
  *tflops = 2.0 * fmas / (static_cast<double>(best) * 1e-3) / 1e12;
  return PES_OK;
}

extern "C" pes_status pes_int_peak(int32_t repeats, double* tops) {
  if (!tops) return fail(PES_EINVAL, "tops is NULL");
  int dev = 0, nsm = 0;
  PES_CUDA(cudaGetDevice(&dev));
  PES_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  long long* sink = nullptr;
  const int threads = 256, blocks = nsm * 4, iters = 8192;
  PES_CUDA(cudaMalloc(&sink, sizeof(long long) * static_cast<size_t>(blocks)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  pes::launch_int_peak(sink, blocks, threads, iters / 8, nullptr);
  for (int r = 0; r < std::max(1, repeats); ++r) {
    cudaEventRecord(e0, nullptr);
    pes::launch_int_peak(sink, blocks, threads, iters, nullptr);
    cudaEventRecord(e1, nullptr);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "int peak kernel");
  *tops = static_cast<double>(blocks) * threads * iters * 64.0 / (static_cast<double>(best) * 1e-3) / 1e12;
  return PES_OK;
}

// ---------------------------------------------------------------------------
// job compiler introspection
// ---------------------------------------------------------------------------

extern "C" pes_status pes_jobc_stats(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                                     int32_t paper_layout, int64_t* stats, int32_t* layer_sizes, int32_t cap) {
  return pes_jobc_stats_powers(supp_ptr, supp_idx, nullptr, N, n, paper_layout, stats, layer_sizes, cap);
}

extern "C" pes_status pes_jobc_stats_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                            int32_t N, int32_t n, int32_t paper_layout, int64_t* stats,
                                            int32_t* layer_sizes, int32_t cap) {
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, N, n, sup, supp_exp);
  if (s != PES_OK) return s;
  if (paper_layout && !sup.ex.empty()) return fail(PES_EINVAL, "the paper's data array has no powers");
  pes::Program1 G = pes::compile(sup, 0, paper_layout != 0, paper_layout == 0);
  std::vector<int64_t> lv = pes::paper_add_levels(sup);
  if (stats) {
    int64_t paper_adds = 0;
    for (int64_t v : lv) paper_adds += v;
    stats[0] = static_cast<int64_t>(G.jobs.size());
    stats[1] = G.n_layers;
    stats[2] = static_cast<int64_t>(G.add_src.size());
    stats[3] = paper_adds;
    stats[4] = G.n_slots;
    stats[5] = static_cast<int64_t>(lv.size());
    stats[6] = paper_layout ? 0 : G.vjp_fwd_jobs - static_cast<int64_t>(G.jobs.size());
    stats[7] = paper_layout ? 0 : static_cast<int64_t>(G.vjp_jobs.size()) - G.vjp_fwd_jobs;
  }
  if (layer_sizes)
    for (int32_t L = 1; L <= G.n_layers && L <= cap; ++L)
      layer_sizes[L - 1] = G.layer_ptr[static_cast<size_t>(L)] - G.layer_ptr[static_cast<size_t>(L) - 1];
  return PES_OK;
}

extern "C" pes_status pes_jobc_jobs(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                                    int32_t paper_layout, int32_t* jobs, int64_t cap) {
  return pes_jobc_jobs_powers(supp_ptr, supp_idx, nullptr, N, n, paper_layout, jobs, cap);
}

extern "C" pes_status pes_jobc_jobs_powers(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                           int32_t N, int32_t n, int32_t paper_layout, int32_t* jobs, int64_t cap) {
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, N, n, sup, supp_exp);
  if (s != PES_OK) return s;
  if (paper_layout && !sup.ex.empty()) return fail(PES_EINVAL, "the paper's data array has no powers");
  pes::Program1 G = pes::compile(sup, 0, paper_layout != 0, false);
  for (size_t t = 0; t < G.jobs.size() && static_cast<int64_t>(t) < cap; ++t) {
    jobs[4 * t + 0] = G.jobs[t].in1;
    jobs[4 * t + 1] = G.jobs[t].in2;
    jobs[4 * t + 2] = G.jobs[t].out;
    jobs[4 * t + 3] = G.jobs[t].layer;
  }
  return PES_OK;
}

extern "C" pes_status pes_jobc_program(const int32_t* supp_ptr, const int32_t* supp_idx, const int32_t* supp_exp,
                                       int32_t N, int32_t n, int32_t complex_series, int32_t P,
                                       const int32_t* poly_ptr, int32_t with_vjp, int64_t* counts, int32_t* jobs,
                                       int32_t* add_ptr, int32_t* add_src, int32_t* add_mult) {
  if (!counts) return fail(PES_EINVAL, "counts is NULL");
  if (P > 0 && complex_series) return fail(PES_EINVAL, "systems are real");
  if (P > 0) {
    if (!poly_ptr || poly_ptr[0] != 0 || poly_ptr[P] != N) return fail(PES_EINVAL, "bad poly_ptr");
    if (static_cast<int64_t>(P) * (n + 1) >= (1LL << 30)) return fail(PES_EINVAL, "too many outputs");
    for (int32_t p = 0; p < P; ++p)
      if (poly_ptr[p + 1] < poly_ptr[p]) return fail(PES_EINVAL, "poly_ptr must not decrease");
  }
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, N, n, sup, supp_exp);
  if (s != PES_OK) return s;
  pes::Program1 G = P > 0 ? pes::compile_system(sup, std::vector<int32_t>(poly_ptr, poly_ptr + P + 1), 0,
                                                with_vjp != 0)
                          : pes::compile(sup, 0, false, with_vjp != 0);
  if (complex_series) G = pes::complexify(G);
  counts[0] = static_cast<int64_t>(G.jobs.size());
  counts[1] = static_cast<int64_t>(G.add_ptr.size()) - 1;
  counts[2] = static_cast<int64_t>(G.add_src.size());
  counts[3] = with_vjp ? G.n_slots_vjp : G.n_slots;
  counts[4] = static_cast<int64_t>(G.vjp_jobs.size());
  counts[5] = G.vjp_fwd_jobs;
  counts[6] = G.slot_u;
  counts[7] = G.slot_g0;
  counts[8] = G.slot_r0;
  counts[9] = G.n_input_slots;
  counts[10] = G.const0;
  counts[11] = G.slot_up0;
  counts[12] = G.slot_J0;
  counts[13] = G.slot_rJ0;
  auto put_job = [&](size_t t, const pes::ConvJob& j) {
    jobs[5 * t + 0] = j.in1;
    jobs[5 * t + 1] = j.in2;
    jobs[5 * t + 2] = j.out;
    jobs[5 * t + 3] = j.layer;
    jobs[5 * t + 4] = j.kind;
  };
  if (jobs) {
    for (size_t t = 0; t < G.jobs.size(); ++t) put_job(t, G.jobs[t]);
    for (size_t t = 0; t < G.vjp_jobs.size(); ++t) put_job(G.jobs.size() + t, G.vjp_jobs[t]);
  }
  if (add_ptr) std::memcpy(add_ptr, G.add_ptr.data(), G.add_ptr.size() * sizeof(int32_t));
  if (add_src) std::memcpy(add_src, G.add_src.data(), G.add_src.size() * sizeof(int32_t));
  if (add_mult) std::memcpy(add_mult, G.add_mult.data(), G.add_mult.size() * sizeof(int32_t));
  return PES_OK;
}

extern "C" pes_status pes_jobc_add_levels(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                                          int64_t* levels, int32_t cap, int32_t* nlevels) {
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, N, n, sup);
  if (s != PES_OK) return s;
  std::vector<int64_t> lv = pes::paper_add_levels(sup);
  if (nlevels) *nlevels = static_cast<int32_t>(lv.size());
  for (size_t t = 0; t < lv.size() && static_cast<int32_t>(t) < cap; ++t) levels[t] = lv[t];
  return PES_OK;
}

extern "C" pes_status pes_jobc_add_terms(const int32_t* supp_ptr, const int32_t* supp_idx, int32_t N, int32_t n,
                                         int32_t* add_ptr, int32_t* add_src, int64_t cap) {
  return pes_jobc_add_terms_powers(supp_ptr, supp_idx, nullptr, N, n, add_ptr, add_src, nullptr, cap);
}

extern "C" pes_status pes_jobc_add_terms_powers(const int32_t* supp_ptr, const int32_t* supp_idx,
                                                const int32_t* supp_exp, int32_t N, int32_t n, int32_t* add_ptr,
                                                int32_t* add_src, int32_t* add_mult, int64_t cap) {
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, N, n, sup, supp_exp);
  if (s != PES_OK) return s;
  pes::Program1 G = pes::compile(sup, 0, false, false);
  if (add_ptr) std::memcpy(add_ptr, G.add_ptr.data(), G.add_ptr.size() * sizeof(int32_t));
  for (size_t t = 0; t < G.add_src.size() && static_cast<int64_t>(t) < cap; ++t) {
    if (add_src) add_src[t] = G.add_src[t];
    if (add_mult) add_mult[t] = G.add_mult[t];
  }
  return PES_OK;
}

extern "C" pes_status pes_jobc_add_terms_system(int32_t P, const int32_t* poly_ptr, const int32_t* supp_ptr,
                                                const int32_t* supp_idx, const int32_t* supp_exp, int32_t n,
                                                int32_t* const0, int32_t* add_ptr, int32_t* add_src,
                                                int32_t* add_mult, int64_t cap) {
  if (P < 1 || !poly_ptr || poly_ptr[0] != 0) return fail(PES_EINVAL, "bad poly_ptr");
  if (n < 1 || static_cast<int64_t>(P) * (n + 1) >= (1LL << 30))
    return fail(PES_EINVAL, "P x (n + 1) outputs must stay below 2^30");
  for (int32_t p = 0; p < P; ++p)
    if (poly_ptr[p + 1] < poly_ptr[p]) return fail(PES_EINVAL, "poly_ptr must not decrease");
  pes::Supports sup;
  pes_status s = build_supports(supp_ptr, supp_idx, poly_ptr[P], n, sup, supp_exp);
  if (s != PES_OK) return s;
  pes::Program1 G = pes::compile_system(sup, std::vector<int32_t>(poly_ptr, poly_ptr + P + 1), 0);
  if (const0) *const0 = G.const0;
  if (add_ptr) std::memcpy(add_ptr, G.add_ptr.data(), G.add_ptr.size() * sizeof(int32_t));
  for (size_t t = 0; t < G.add_src.size() && static_cast<int64_t>(t) < cap; ++t) {
    if (add_src) add_src[t] = G.add_src[t];
    if (add_mult) add_mult[t] = G.add_mult[t];
  }
  return PES_OK;
}

extern "C" pes_status pes_selftest_timeout(int64_t timeout_ms, int32_t* device_status) {
  if (timeout_ms <= 0 || timeout_ms > 60000) return fail(PES_EINVAL, "timeout_ms must be in (0, 60000]");
  // one monomial x_0 of degree 0: a single job, made to wait on its own flag,
  // once in the whole-series kernel and once in the tiled kernel
  const int32_t ptr[2] = {0, 1}, idx[1] = {0};
  pes_status st = PES_OK;
  for (int32_t tile : {0, 16}) {
    pes_options o;
    pes_default_options(&o);
    o.with_vjp = 0;
    o.timeout_ms = timeout_ms;
    o.tile = tile;
    pes_plan_t P = nullptr;
    pes_status s = pes_plan_ex(ptr, idx, 1, 1, 0, 1, &o, &P);
    if (s != PES_OK) return s;
    std::unique_ptr<pes_plan_s> guard(P);
    std::vector<pes::ConvJob> jobs = P->prog.jobs;
    jobs[0].dep1 = 0;  // the job waits for itself: the flag is never set
    JobList L;
    s = P->ex.make_joblist(L, jobs);
    if (s != PES_OK) return s;
    PES_CUDA(pes::launch_prologue(P->ex.ctrl, nullptr));
    PES_CUDA(P->ex.run_dag(L, 0, nullptr));
    st = P->ex.check(nullptr);
    if (st != PES_ETIMEOUT) break;
  }
  if (device_status) *device_status = static_cast<int32_t>(st);
  return st == PES_ETIMEOUT ? PES_OK : fail(PES_EINTERNAL, "the wait did not report a timeout");
}

extern "C" const char* pes_status_string(pes_status s) {
  switch (s) {
    case PES_OK: return "PES_OK";
    case PES_EINVAL: return "PES_EINVAL: invalid argument";
    case PES_EUNSUPPORTED_K: return "PES_EUNSUPPORTED_K: k must be 1,2,3,4,5,8 or 10";
    case PES_ENOMEM: return "PES_ENOMEM: allocation failed";
    case PES_ECUDA: return "PES_ECUDA: CUDA runtime error";
    case PES_ETIMEOUT: return "PES_ETIMEOUT: a device-side wait gave up";
    case PES_EINTERNAL: return "PES_EINTERNAL: internal error";
    case PES_EUNSUPPORTED_SIZE: return "PES_EUNSUPPORTED_SIZE: degree too large";
    default: return "unknown pes_status";
  }
}

extern "C" const char* pes_last_error(void) { return g_last_error.c_str(); }

namespace pes {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace pes
