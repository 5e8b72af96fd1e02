// kernels.hpp -- launch interface between the C-ABI layer and the CUDA kernels.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "jobc.hpp"

namespace pes {

// Arithmetic of the convolution multiply-accumulate loop.
enum : int32_t {
  ARITH_FP64 = 0,  // digit products accumulated with FP64 FMA (exact, flushed every R terms)
  ARITH_INT = 1,   // digit products accumulated with 32x32->64-bit integer multiply-add
};

// Per-plan control block in device memory.
struct Ctrl {
  int32_t epoch;      // incremented once per call by the prologue kernel
  int32_t abort;      // set when any wait gives up
  int32_t status;     // first error code (pes_status), 0 when fine
  int32_t pad0;
  int32_t next[4];    // job dispatch counters (one per DAG launch of a call)
  long long diag[4];  // diagnostics: [0] job that timed out, [1] waiting job
};

// The workspace holds every series in digit form (see InstInfo): int32 words.
struct DagArgs {
  const ConvJob* jobs;
  int32_t njobs;
  int32_t counter;          // which Ctrl::next
  int32_t* flags;           // per job: epoch when done
  const InstInfo* inst;
  int32_t* ws;
  Ctrl* ctrl;
  int32_t smax;             // largest padded stride of the instances
  int32_t dmax;             // largest degree
  int32_t depth;            // staging depth: 1, or 2 (next job staged while this one is rounded)
  int32_t split;            // parts per job (integer variant: 1 to 16, a power of two): part p of job j is
                            // dispatched, flagged and waited for as j * split + p
  long long timeout_ns;     // bound on every wait
  int32_t tile;             // > 0: the tiled kernel, output tiles of `tile` coefficients, `split`
                            // tiles per job (sub-job j * split + t is tile t of job j)
};

struct AddArgs {
  const AddOut* outs;
  int32_t nouts;
  int32_t to_ws;            // 1: results in digit form into workspace slot dst_off of the instance
  const int64_t* item_ptr;  // nouts + 1 prefix sums of (d + 1) over outputs
  const int32_t* contrib;
  const int32_t* mult;      // integer factor of every contribution (nullptr: all 1)
  const InstInfo* inst;
  int32_t* ws;
  double* dst[2];           // k-limb results: caller buffers by selector
  int32_t group_warps;      // warps that share one output coefficient (1, 2, 4 or 8)
  // Partial sums of a polynomial split over ranks (real single plans; output o
  // of the value is 0, of d p / d x_i is 1 + i, coefficient j of output o is
  // item o (d + 1) + j):
  //   mode 0: round every sum (or write it in digit form, to_ws);
  //   mode 1: write the largest grid of each item's contributions to grid_io;
  //   mode 2: sum each item's contributions on the grid grid_io gives (the
  //           largest over all ranks) and write the L exact digit sums,
  //           unrounded, to acc_out[item * L + p].
  int32_t mode;
  int32_t* grid_io;
  long long* acc_out;
};

// Rounding of digit sums (mode 2 of the addition stage, summed over ranks).
struct RoundArgs {
  const int32_t* grids;     // [(n+1)(d+1)]
  const long long* acc;     // [(n+1)(d+1)][L]
  double* value;            // [k][d+1]
  double* grad;             // [k][n][d+1]
  int32_t n, d;
};

struct CopyArgs {
  const CopyRow* rows;
  int32_t nrows;
  const InstInfo* inst;
  int32_t* ws;
  const double* src[4];  // pack: caller buffers by selector
  double* dst[4];        // unpack: caller buffers by selector
};

// Threads per CTA of the DAG kernel: at least one lane per coefficient pair of
// the largest degree; the register budget of each k caps it.  At k = 10 the cap
// is 256 with two CTAs per SM guaranteed, which holds the kernel to 128
// registers per thread (the multiply-accumulate loop keeps 21 64-bit
// accumulators and a digit row in registers).
__host__ __device__ constexpr int dag_max_threads(int k) { return k >= 10 ? 256 : k >= 8 ? 384 : k >= 4 ? 512 : 768; }
__host__ __device__ constexpr int dag_min_ctas(int k) { return k >= 10 ? 2 : 1; }
// More CTAs per SM at low k keep more jobs in flight while others stage or
// round.  The whole-series kernel's integer variant caps its registers at 64
// for k = 3 (four CTAs of 256 threads per SM) and at 80 for k = 4, 5 (three);
// at k <= 2 a second instantiation for CTAs of at most 256 threads declares
// four CTAs per SM in its launch bounds (measured faster at k <= 2 than the
// same register count reached through a cap), and CTAs wider than that (large
// degrees) take the uncapped kernel.  The accumulators of L <= 12 digits fit
// without spilling.
__host__ __device__ constexpr int dag_max_regs(int k, bool intv) {
  return !intv ? 255 : k <= 2 ? 255 : k <= 3 ? 64 : k <= 5 ? 80 : 255;
}
__host__ __device__ constexpr bool dag_has_narrow(int k, bool intv) { return intv && k <= 2; }
constexpr int kNarrowThreads = 256;  // widest CTA of the narrow instantiation
constexpr int kNarrowCtas = 4;       // CTAs per SM its launch bounds declare
constexpr int kMaxSplit = 16;  // largest number of parts a convolution job is split into

// Shared-memory footprint of the DAG kernel for (k, arith, smax, dmax) at
// staging depth 1 or 2 with `threads` threads per CTA (the integer variant
// keeps one exchange row per thread).
size_t dag_smem_bytes(int k, int arith, int smax, int dmax, int depth, int threads);
// Shared-memory footprint of the tiled DAG kernel (degrees whose whole series
// do not fit) for output tiles of `tile` coefficients, any degree.
size_t dag_tiled_smem_bytes(int k, int arith, int tile);
constexpr int kDefaultTile = 128;  // coefficients per output tile of the tiled kernel
constexpr int kMaxDegree = 16383;  // largest degree the API accepts
int digits_of_k(int k, int arith);
// int32 words of one workspace row (the digits of one coefficient, padded) and
// of one workspace slot (a series of S coefficients: S rows, then S grids).
int ws_row_words(int k, int arith);
inline int64_t ws_slot_words(int k, int arith, int32_t S) {
  return static_cast<int64_t>(S) * (ws_row_words(k, arith) + 1);
}

// Warps of the addition kernel that share one output coefficient, from the
// largest number of contributions of an output: one warp up to 1024 (the
// block barriers of a group cost more than they save below that), then up to
// 8 warps for the long sums (the value of a polynomial of thousands of
// monomials would otherwise be a serial tail of one warp per coefficient).
inline int32_t add_group_warps(int64_t max_contrib) {
  return max_contrib > 4096 ? 8 : max_contrib > 2048 ? 4 : max_contrib > 1024 ? 2 : 1;
}
// The same for a launch of `items` output coefficients on `nsm` SMs: a table
// too small to fill the GPU with one group per coefficient (a few hundred
// coefficients, each a sum of hundreds of contributions) is latency-bound on
// its longest sum, so its groups are widened while the launch stays within 16
// warps per SM and every lane keeps at least two contributions.
inline int32_t add_group_warps(int64_t max_contrib, int64_t items, int32_t nsm) {
  int32_t gw = add_group_warps(max_contrib);
  while (gw < 8 && items * gw * 2 <= 16LL * nsm && max_contrib > 64LL * gw) gw *= 2;
  return gw;
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_prologue(Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_pack(const CopyArgs& a, int k, int arith, cudaStream_t st);
cudaError_t launch_unpack(const CopyArgs& a, int k, int arith, cudaStream_t st);
cudaError_t launch_dag(const DagArgs& a, int k, int arith, int threads, int grid, cudaStream_t st);
cudaError_t launch_add(const AddArgs& a, int k, int arith, int64_t items, cudaStream_t st);
// Two parts of one addition stage, both with groups of 2, 4 or 8 warps per
// output coefficient, in one launch.
cudaError_t launch_add_pair(const AddArgs& a0, int64_t items0, const AddArgs& a1, int64_t items1, int k,
                            int arith, cudaStream_t st);
cudaError_t launch_round_sums(const RoundArgs& a, int k, int arith, cudaStream_t st);
// The same rounding on the host (no GPU needed).
int round_sums_host(int k, int arith, const RoundArgs& a);
cudaError_t dag_occupancy(int k, int arith, int threads, size_t smem, int* blocks_per_sm, bool tiled = false);
cudaError_t dag_prepare(int k, int arith, size_t smem, bool tiled = false);
cudaError_t launch_md_binary(int op, int k, const double* x, const double* y, double* out,
                             int64_t count, cudaStream_t st);
cudaError_t launch_fp64_peak(double* sink, int blocks, int threads, int iters, cudaStream_t st);
cudaError_t launch_int_peak(long long* sink, int blocks, int threads, int iters, cudaStream_t st);

}  // namespace pes
