// kernels.cu -- the CUDA kernels of the evaluation and differentiation path.
//
//   pack      caller series -> workspace (padded limb planes)        (Sec. 2, data layout)
//   dag       all convolution jobs of all layers in one persistent launch (Sec. 5):
//             operands staged into shared memory by TMA bulk copies, converted
//             to exact digits, every output coefficient the exact sum of its
//             terms (Eq. eqconvform) rounded once to k limbs
//   add       value and gradient sums (Sec. 5, addition jobs): one warp per
//             output coefficient, contributions spread over the lanes, exact
//             digit sums reduced with warp shuffles
//   unpack    workspace -> caller series
//   md_binary elementwise k-double add / mul (Sec. 1 arithmetic)
//   fp64_peak DFMA throughput microbenchmark (the roofline of the FP64 variant)
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "digits.cuh"
#include "kernels.hpp"
#include "md.cuh"

namespace pes {

namespace {

constexpr int kStatusTimeout = 5;  // PES_ETIMEOUT

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Mark a sub-job done.  Every thread of the CTA stored its output rows before
// the block barrier that precedes this call, and the barrier makes those
// stores visible to the calling thread; the release store is cumulative over
// them, so a CTA that reads the flag with an acquire load sees the rows.  The
// proxy fence orders the rows (written through the generic proxy) before the
// bulk copies a consumer issues after it has seen the flag.
__device__ __forceinline__ void publish_flag(int32_t* flag, int epoch) {
  fence_proxy_async_global();
  st_release(flag, epoch);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Plain (non-tensor, non-multicast) bulk copy global -> this CTA's shared memory.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long timeout_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  unsigned long long t0 = global_timer();
  for (;;) {
    if (mbar_try_wait(bar, phase)) return true;
    if (static_cast<long long>(global_timer() - t0) > timeout_ns) return false;
  }
}

// A 64-bit two's-complement accumulator of the integer pipe, kept as two
// 32-bit words: a digit product x * y (a signed 64-bit value) is added as a
// 32-bit multiply-add of its low word with carry-out, then a multiply-add of
// its high word with carry-in.  The sum is the same 64-bit value a 64-bit
// multiply-add gives; this form needs one heavy-pipe instruction per product
// and no extra 64-bit addition on the ALU.
struct Acc64 {
  uint32_t lo;
  int32_t hi;
};

// acc += x * y, exactly: 32x32 -> 64-bit integer multiply-add in place, or FP64 FMA
// on digit products that are exact by construction.
__device__ __forceinline__ void mac(int32_t x, int32_t y, Acc64& acc) {
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.s32 %1, %2, %3, %1;" : "+r"(acc.lo), "+r"(acc.hi) : "r"(x), "r"(y));
}

__device__ __forceinline__ void mac(double x, double y, double& acc) { acc = __fma_rn(x, y, acc); }

__device__ __forceinline__ void acc_clear(Acc64& a) {
  a.lo = 0u;
  a.hi = 0;
}
__device__ __forceinline__ void acc_clear(double& a) { a = 0.0; }
__device__ __forceinline__ long long acc_value(const Acc64& a) {
  return static_cast<long long>((static_cast<unsigned long long>(static_cast<uint32_t>(a.hi)) << 32) | a.lo);
}
__device__ __forceinline__ long long acc_value(double a) { return __double2ll_rn(a); }

__device__ __forceinline__ void set_error(Ctrl* ctrl, int code, long long d0, long long d1) {
  if (atomicCAS(&ctrl->status, 0, code) == 0) {
    ctrl->diag[0] = d0;
    ctrl->diag[1] = d1;
  }
  atomicExch(&ctrl->abort, 1);
}

// Parts of every job of the launch (a split of 0 reads as 1).
__device__ __forceinline__ int parts(const DagArgs& a) { return a.split > 1 ? a.split : 1; }

// Every part of job `dep` of this call has completed (dep < 0: an input series).
__device__ __forceinline__ bool is_done(const DagArgs& a, int dep, int epoch) {
  if (dep < 0) return true;
  const int s = parts(a);
  for (int p = 0; p < s; ++p)
    if (ld_acquire(a.flags + dep * s + p) != epoch) return false;
  return true;
}

// Bounded wait until sub-job `f` (a flag index) of this call has completed.
__device__ bool wait_flag(const DagArgs& a, int f, int epoch, int job) {
  if (ld_acquire(a.flags + f) == epoch) return true;
  unsigned long long t0 = global_timer();
  for (;;) {
    if (ld_acquire(a.flags + f) == epoch) return true;
    if (*reinterpret_cast<volatile int32_t*>(&a.ctrl->abort)) return false;
    if (static_cast<long long>(global_timer() - t0) > a.timeout_ns) {
      set_error(a.ctrl, kStatusTimeout, f, job);
      return false;
    }
    __nanosleep(200);
  }
}

// Bounded wait until every part of job `dep` of this call has completed.
__device__ bool wait_done(const DagArgs& a, int dep, int epoch, int job) {
  if (dep < 0) return true;
  const int s = parts(a);
  for (int p = 0; p < s; ++p)
    if (!wait_flag(a, dep * s + p, epoch, job)) return false;
  return true;
}

// ---------------------------------------------------------------------------
// DAG kernel shared-memory layout
// ---------------------------------------------------------------------------

struct DagLayout {
  size_t raw, exch, xdig, ydig, gx, gy, gs, bar, misc, total;
};

// Row strides of the digit arrays (in digits).  Integer variant: an X row is L
// zero digits followed by the L digits (so a term shifted by delta digits reads
// the row delta digits early without any select), odd stride; a Y row is padded
// to a multiple of 4 digits with an odd number of 16-byte groups, so it is read
// with 128-bit loads without bank conflicts.  FP64 variant: odd stride L | 1.
__host__ __device__ constexpr int x_stride(int L, bool intv) { return intv ? 2 * L + 1 : (L | 1); }
__host__ __device__ constexpr int y_stride(int L, bool intv) {
  return intv ? (((L + 3) / 4) % 2 == 1 ? (L + 3) / 4 * 4 : (L + 3) / 4 * 4 + 4) : (L | 1);
}

// Staging depth 1: the staged limb planes of a job share their bytes with the
// exchange rows (the limbs are converted to digits before the rows are
// zeroed).  Depth 2: separate buffers, so that the next job's operands can be
// staged while the exchange rows of the current one are still being rounded.
//
// Exchange rows of the integer variant: one private row per lane of the CTA
// and one extra row per coefficient-pair group (for the one lane of a group
// whose run crosses from the short to the long coefficient), each L + 1
// 64-bit words at an odd stride in 8-byte units (private_row_stride), so that
// every row has a single writer and no shared-memory atomics are needed.  The
// FP64 variant keeps one row per output coefficient, updated atomically.
// int32 words per workspace row of one coefficient: the integer variant's Y
// row stride (so that a whole operand series lands as Y rows with one bulk
// copy), else the digits rounded up to 16 bytes.
__host__ __device__ constexpr int row_words(int L, bool intv) { return intv ? y_stride(L, true) : (L + 3) / 4 * 4; }

__host__ __device__ constexpr int private_row_stride(int L) { return (L + 1) | 1; }
// coefficient-pair groups of a series of degree d: (d+1)/2 pairs (j, d-j),
// j < d-j, and the middle coefficient d/2 alone when d+1 is odd
__host__ __device__ constexpr int pair_groups(int d) { return (d + 2) / 2; }

__host__ __device__ inline DagLayout dag_layout(int K, int L, bool intv, int smax, int dmax, int depth, int threads) {
  const int digit_bytes = intv ? 4 : 8;
  DagLayout o;
  // staged digit rows: X only (Y rows land in place) for the integer variant,
  // X and Y for the FP64 variant (converted to doubles)
  size_t raw_bytes = size_t(intv ? 1 : 2) * smax * row_words(L, intv) * sizeof(int32_t);
  size_t exch_bytes = intv ? size_t(threads + pair_groups(dmax)) * private_row_stride(L) * sizeof(unsigned long long)
                           : size_t(dmax + 1) * (L + 1) * sizeof(unsigned long long);
  size_t off = 0;
  o.raw = 0;
  if (depth >= 2) {
    o.exch = align_up(raw_bytes, 128);
    off = align_up(o.exch + exch_bytes, 128);
  } else {
    o.exch = 0;
    off = align_up(raw_bytes > exch_bytes ? raw_bytes : exch_bytes, 128);
  }
  o.xdig = off;
  off = align_up(off + size_t(smax) * x_stride(L, intv) * digit_bytes, 16);
  o.ydig = off;
  off = align_up(off + size_t(smax) * y_stride(L, intv) * digit_bytes, 16);
  o.gx = off;
  off += size_t(smax) * 4;
  o.gy = off;
  off += size_t(smax) * 4;
  o.gs = off;
  off = align_up(off + size_t(smax) * 4, 16);
  o.bar = off;
  off += 16;
  o.misc = off;
  off += 64;
  o.total = align_up(off, 128);
  return o;
}

// first coefficient j with start(j) > g, minus one
__device__ __forceinline__ long long conv_start(long long j) { return j * (j + 1) / 2; }
__device__ __forceinline__ long long corr_start(long long j, long long d) { return j * (d + 1) - j * (j - 1) / 2; }

// The multiply-accumulate of one term into L accumulators and the flush of the
// accumulators into an exchange row, shared by the whole-series and the tiled
// convolution kernels.
template <int K, bool INTV>
struct DigitMac {
  using DigitT = typename std::conditional<INTV, int32_t, double>::type;
  using AccT = typename std::conditional<INTV, Acc64, double>::type;
  static constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  static constexpr int L = digits_for_k(K, B);
  static constexpr int XS = x_stride(L, INTV);
  static constexpr int YS = y_stride(L, INTV);
  static constexpr int XOFF = INTV ? L : 0;  // digits start after the zero prefix

  // acc += the term x_ix * y_iy of an output coefficient whose grid lies delta
  // digits above the term's: the products of digits p of x and q of y with
  // p + delta + q < L (digit positions below the grid's L digits are dropped).
  // The reference grid is the largest of the coefficient's terms, so delta >= 0;
  // the unsigned compare also skips a negative delta, which would address
  // outside the X row.
  __device__ __forceinline__ static void term(const DigitT* xdig, const DigitT* ydig, int ix, int iy, int delta,
                                              AccT (&A)[L]) {
    if constexpr (INTV) {
      if (static_cast<unsigned>(delta) < static_cast<unsigned>(L)) {
        // zero prefix: digit p of the shifted term is xs[p], no select
        const int32_t* xs = xdig + ix * XS + XOFF - delta;
        const int4* y4 = reinterpret_cast<const int4*>(ydig + iy * YS);
        int32_t Y[YS];
#pragma unroll
        for (int v = 0; v < YS / 4; ++v) {
          const int4 t4 = y4[v];
          Y[4 * v] = t4.x;
          Y[4 * v + 1] = t4.y;
          Y[4 * v + 2] = t4.z;
          Y[4 * v + 3] = t4.w;
        }
#pragma unroll
        for (int p = 0; p < L; ++p) {
          const int32_t xv = xs[p];
#pragma unroll
          for (int q = 0; q < L - p; ++q) mac(xv, Y[q], A[p + q]);
        }
      }
    } else {
      if (static_cast<unsigned>(delta) < static_cast<unsigned>(L)) {
        const DigitT* yr = ydig + iy * YS;
        const DigitT* xr = xdig + ix * XS;
        DigitT Y[L];
#pragma unroll
        for (int q = 0; q < L; ++q) Y[q] = yr[q];
#pragma unroll
        for (int p = 0; p < L; ++p) {
          const int id = p - delta;
          DigitT xv = xr[id < 0 ? 0 : id];
          xv = id < 0 ? DigitT(0) : xv;
#pragma unroll
          for (int q = 0; q < L - p; ++q) mac(xv, Y[q], A[p + q]);
        }
      }
    }
  }

  // Add the accumulators into an exchange row (L + 1 words of 8 bytes): A[t]
  // belongs to word t+1 (word 0 is headroom above the grid's top digit).  One
  // flush may carry up to 2^63 per accumulator, so the values are first carried
  // in registers: word t+1 takes the low B bits of A[t] plus the part of A[t+1]
  // above its low B bits, word 0 the part of A[0] above B bits, so no word takes
  // more than 2^36 in magnitude per flush.  Each such contribution w is added as
  // two 32-bit integers, w = h 2^18 + l with l in [-2^17, 2^17): h into the first
  // half of the word and l into the second, with native 32-bit shared-memory
  // atomic adds (a 64-bit shared-memory atomic add is a compare-and-swap loop,
  // and the lanes of a coefficient group flush the same words at the same
  // step).  Both halves stay exact for 2^13 flushes into one word, far more than
  // any coefficient receives (its terms / R flushes plus two per lane); the
  // word's value is h 2^18 + l (exch_word).
  __device__ __forceinline__ static void flush(unsigned long long* row, AccT (&A)[L]) {
    int32_t* r32 = reinterpret_cast<int32_t*>(row);
    long long hi_next = 0;  // part of A[t+1] above its low B bits
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      const long long v = acc_value(A[t]);
      const long long w = (v & ((1LL << B) - 1)) + hi_next;
      hi_next = v >> B;  // arithmetic shift: v = hi * 2^B + lo
      add_split(r32 + 2 * (t + 1), w);
      acc_clear(A[t]);
    }
    add_split(r32, hi_next);
  }

  // The same carried contributions added into a row that only this thread
  // writes (plain 64-bit loads and stores; each word takes at most 2^36 per
  // flush, far inside 64 bits).
  __device__ __forceinline__ static void flush_own(unsigned long long* row, AccT (&A)[L]) {
    long long* r64 = reinterpret_cast<long long*>(row);
    long long hi_next = 0;
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      const long long v = acc_value(A[t]);
      const long long w = (v & ((1LL << B) - 1)) + hi_next;
      hi_next = v >> B;
      r64[t + 1] += w;
      acc_clear(A[t]);
    }
    r64[0] += hi_next;
  }

  // row[0..1] += w as h 2^18 + l, l in [-2^17, 2^17)
  __device__ __forceinline__ static void add_split(int32_t* row, long long w) {
    if (w == 0) return;
    const long long l = ((w + (1LL << 17)) & ((1LL << 18) - 1)) - (1LL << 17);
    const long long h = (w - l) >> 18;
    if (h != 0) atomicAdd(row, static_cast<int32_t>(h));
    if (l != 0) atomicAdd(row + 1, static_cast<int32_t>(l));
  }
};

// Value of exchange-row word t (two 32-bit halves h, l: h 2^18 + l).
__device__ __forceinline__ int64_t exch_word(const unsigned long long* row, int t) {
  const int2 p = reinterpret_cast<const int2*>(row)[t];
  return static_cast<int64_t>(p.x) * (1LL << 18) + p.y;
}

template <int K, bool INTV, bool NARROW = false>
__global__ void __launch_bounds__(NARROW ? kNarrowThreads : dag_max_threads(K),
                                  NARROW ? kNarrowCtas : (INTV ? dag_min_ctas(K) : 1))
    __maxnreg__(NARROW ? 255 : dag_max_regs(K, INTV)) dag_kernel(DagArgs a) {
  using DigitT = typename std::conditional<INTV, int32_t, double>::type;
  using AccT = typename DigitMac<K, INTV>::AccT;
  constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  constexpr int L = digits_for_k(K, B);
  constexpr int XS = x_stride(L, INTV);
  constexpr int YS = y_stride(L, INTV);
  constexpr int XOFF = INTV ? L : 0;  // digits start after the zero prefix
  constexpr int RW = row_words(L, INTV);  // int32 words per workspace row
  // accumulators stay exact for R terms (each term adds at most L products of
  // magnitude 2^(2B-2)): 2^53 for FP64, 2^63 for int64
  constexpr int R = INTV ? static_cast<int>((1LL << (63 - 2 * (B - 1))) / L) : 128 / L;

  extern __shared__ __align__(128) unsigned char smem[];
  const DagLayout lay = dag_layout(K, L, INTV, a.smax, a.dmax, a.depth, blockDim.x);
  int32_t* raw = reinterpret_cast<int32_t*>(smem + lay.raw);
  unsigned long long* exch = reinterpret_cast<unsigned long long*>(smem + lay.exch);
  DigitT* xdig = reinterpret_cast<DigitT*>(smem + lay.xdig);
  DigitT* ydig = reinterpret_cast<DigitT*>(smem + lay.ydig);
  int32_t* gx = reinterpret_cast<int32_t*>(smem + lay.gx);
  int32_t* gy = reinterpret_cast<int32_t*>(smem + lay.gy);
  int32_t* gs = reinterpret_cast<int32_t*>(smem + lay.gs);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + lay.bar);
  int32_t* misc = reinterpret_cast<int32_t*>(smem + lay.misc);

  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const uint32_t bar_addr = smem_u32(bar);
  if (tid == 0) {
    mbar_init(bar_addr, 1);
    fence_mbar_init();
  }
  if constexpr (INTV) {
    // zero prefixes of the X rows (the conversions only write the digit part)
    for (int t = tid; t < a.smax * XS; t += T) xdig[t] = 0;
  }
  __syncthreads();
  const int epoch = *reinterpret_cast<volatile int32_t*>(&a.ctrl->epoch);
  uint32_t phase = 0;
  // Staging depth 2: one thread with no coefficient to round (the last one,
  // when the CTA is wider than the largest series) claims the next job while
  // the others round the current one, and stages it at once if its operands
  // are ready.  It never waits there: the job it would wait for may be the one
  // this CTA has not released yet.  A job claimed but not staged is staged,
  // with a bounded wait, at the top of the next iteration.
  const bool ahead = a.depth >= 2;
  const int stager = (ahead && T > a.dmax + 1) ? T - 1 : 0;

  // A job may be split into `split` parts, each computing the output
  // coefficients of a contiguous range of coefficient pairs; part p of job j is
  // sub-job j * split + p, with a completion flag of its own.
  const int split = parts(a);
  const int nsub = a.njobs * split;

  // misc[0]: claimed sub-job, misc[1]: failure, misc[2]: its operands are being staged
  auto claim = [&]() {
    misc[0] = atomicAdd(&a.ctrl->next[a.counter], 1);
    misc[1] = 0;
    misc[2] = 0;
  };
  // Start the TMA bulk copies of the claimed sub-job's two operand series
  // (digit rows and grids) once both are complete; `blocking`: wait (bounded)
  // for them, else only look.
  auto stage = [&](bool blocking) {
    const int sj = misc[0];
    if (sj >= nsub) return;
    const int job = sj / split;
    const ConvJob jb = a.jobs[job];
    const InstInfo in = a.inst[jb.inst];
    if (INTV && (in.d + 2) / 2 > T) {  // at least one lane per coefficient pair: the plan sizes the CTA
      if (blocking) {
        set_error(a.ctrl, 6, job, in.d);
        misc[1] = 1;
      }
      return;
    }
    if (blocking) {
      if (!wait_done(a, jb.dep1, epoch, job) || !wait_done(a, jb.dep2, epoch, job)) {
        misc[1] = 1;
        return;
      }
    } else if (!is_done(a, jb.dep1, epoch) || !is_done(a, jb.dep2, epoch)) {
      return;
    }
    // digit rows, then grids, of each operand series (int32 words)
    const int32_t* xs = a.ws + in.ws_base + static_cast<long long>(jb.in1) * in.ws_sstride;
    const int32_t* ys = a.ws + in.ws_base + static_cast<long long>(jb.in2) * in.ws_sstride;
    fence_proxy_async_global();
    fence_proxy_async_shared();
    const uint32_t rbytes = static_cast<uint32_t>(in.S) * RW * sizeof(int32_t);
    const uint32_t gbytes = static_cast<uint32_t>(in.S) * sizeof(int32_t);
    mbar_expect_tx(bar_addr, 2u * (rbytes + gbytes));
    bulk_g2s(smem_u32(raw), xs, rbytes, bar_addr);
    if constexpr (INTV) {
      bulk_g2s(smem_u32(ydig), ys, rbytes, bar_addr);
    } else {
      bulk_g2s(smem_u32(raw) + rbytes, ys, rbytes, bar_addr);
    }
    bulk_g2s(smem_u32(gx), xs + static_cast<long long>(in.S) * RW, gbytes, bar_addr);
    bulk_g2s(smem_u32(gy), ys + static_cast<long long>(in.S) * RW, gbytes, bar_addr);
    misc[2] = 1;
  };

  bool claimed = false;  // the stager already claimed the next job
  for (;;) {
    if (tid == 0) {
      if (!claimed) claim();
      if (!misc[2]) stage(true);
    }
    __syncthreads();
    const int sj = misc[0];
    if (sj >= nsub || misc[1]) break;
    const int job = sj / split;
    const int part = sj - job * split;
    const ConvJob jb = a.jobs[job];
    const InstInfo in = a.inst[jb.inst];
    const int d = in.d;
    // Coefficients j and d-j form group min(j, d-j) (the middle coefficient d/2
    // of an even degree is the last group); this part owns groups [g_lo, g_hi).
    const int npairs = (d + 1) / 2;
    const int ngroups = npairs + (((d + 1) & 1) != 0 ? 1 : 0);
    const int g_lo = part * ngroups / split, g_hi = (part + 1) * ngroups / split;
    auto owned = [&](int j) {
      const int g = min(j, d - j);
      return g >= g_lo && g < g_hi;
    };
    const int S = in.S;
    int32_t* zrows = a.ws + in.ws_base + static_cast<long long>(jb.out) * in.ws_sstride;
    int32_t* zgrid = zrows + static_cast<long long>(S) * RW;

    // ---- the operand series (digit rows and grids) land in shared memory ----
    const bool landed = mbar_wait(bar_addr, phase, a.timeout_ns);
    if (!__syncthreads_and(landed)) {
      if (tid == 0) set_error(a.ctrl, kStatusTimeout, job, -2);
      mbar_wait(bar_addr, phase, a.timeout_ns);  // let copies in flight land before exit
      break;
    }
    phase ^= 1u;

    const bool elementwise = jb.kind == JOB_ADD || jb.kind == JOB_SUB;
    if (elementwise) {
      // ---- out = in1 +- in2 coefficient by coefficient, exactly, as L digits ----
      const int32_t* rx = raw;                                  // X rows (stride RW)
      const int32_t* ry = INTV ? reinterpret_cast<const int32_t*>(ydig) : raw + S * RW;  // Y rows
      const long long sgn = jb.kind == JOB_SUB ? -1 : 1;
      for (int j = tid; j <= d; j += T) {
        if (!owned(j)) continue;
        const int32_t g = max(gx[j], gy[j]);
        int32_t o[L];
        int32_t gz = GRID_ZERO;
        if (g < -100000) {
#pragma unroll
          for (int p = 0; p < L; ++p) o[p] = 0;
        } else {
          const int sx = g - gx[j], sy = g - gy[j];  // digits below the common grid's top
          int64_t E[L + 1];
          E[0] = 0;
#pragma unroll
          for (int q = 0; q < L; ++q) {
            const long long xv = q >= sx ? rx[j * RW + q - sx] : 0;
            const long long yv = q >= sy ? ry[j * RW + q - sy] : 0;
            E[q + 1] = xv + sgn * yv;
          }
          gz = sum_to_digits<L, B>(E, g + 1, o);
        }
        int4* dst = reinterpret_cast<int4*>(zrows + static_cast<long long>(j) * RW);
#pragma unroll
        for (int v = 0; v < RW / 4; ++v)
          dst[v] = make_int4(4 * v < L ? o[4 * v] : 0, 4 * v + 1 < L ? o[4 * v + 1] : 0,
                             4 * v + 2 < L ? o[4 * v + 2] : 0, 4 * v + 3 < L ? o[4 * v + 3] : 0);
        zgrid[j] = gz;
      }
      __syncthreads();  // the staged rows are read: the next job may be staged
      if (ahead && tid == stager) {
        claim();
        stage(false);
      }
    } else {
      // ---- staged digit rows into the layouts of the multiply-accumulate loop ----
      if constexpr (INTV) {
        // X rows behind their zero prefix (the Y rows and both grids are in place)
        constexpr int V4 = RW / 4;
        const int4* src = reinterpret_cast<const int4*>(raw);
        for (int t = tid; t < (d + 1) * V4; t += T) {
          const int c = t / V4, v = t - c * V4;
          const int4 q = src[t];
          int32_t* dst = xdig + c * XS + XOFF + 4 * v;
          if (4 * v < L) dst[0] = q.x;
          if (4 * v + 1 < L) dst[1] = q.y;
          if (4 * v + 2 < L) dst[2] = q.z;
          if (4 * v + 3 < L) dst[3] = q.w;
        }
      } else {
        const int32_t* rx = raw;
        const int32_t* ry = raw + S * RW;
        for (int t = tid; t < (d + 1) * L; t += T) {
          const int c = t / L, p = t - c * L;
          xdig[c * XS + p] = static_cast<double>(rx[c * RW + p]);
          ydig[c * YS + p] = static_cast<double>(ry[c * RW + p]);
        }
      }
      __syncthreads();

      // ---- zero the exchange rows, reference grid of every output coefficient ----
      const int rows = INTV ? (T + g_hi - g_lo) * private_row_stride(L) : (d + 1) * (L + 1);
      for (int t = tid; t < rows; t += T) exch[t] = 0ull;
      for (int j = tid; j <= d; j += T) {
        if (!owned(j)) continue;
        int32_t m = 2 * GRID_ZERO;
        if (jb.kind == JOB_CONV) {
          for (int i = 0; i <= j; ++i) m = max(m, gx[i] + gy[j - i]);
        } else {
          for (int i = 0; i <= d - j; ++i) m = max(m, gx[j + i] + gy[i]);
        }
        gs[j] = m;
      }
      __syncthreads();

      // ---- multiply-accumulate ----
      {
        const bool conv = jb.kind == JOB_CONV;
        AccT A[L];
  #pragma unroll
        for (int t = 0; t < L; ++t) acc_clear(A[t]);
        auto flush = [&](int jj) { DigitMac<K, INTV>::flush(exch + jj * (L + 1), A); };
        // one term x_ix * y_iy of output coefficient j, delta digits below its grid
        auto term = [&](int ix, int iy, int delta) { DigitMac<K, INTV>::term(xdig, ydig, ix, iy, delta, A); };
        if constexpr (INTV) {
          // Coefficients j and d-j share d+2 terms (the middle coefficient d/2,
          // when d+1 is odd, forms a group of its own, the last one).  Every lane
          // of the CTA belongs to a group: each group gets Q = T / groups
          // consecutive lanes, and the first T mod groups groups one more, so no
          // lane idles.  The lanes of a group split its terms, walked as: the
          // short coefficient from its first term, then the long one from its last
          // term backwards.  At every step all lanes with the same rank q inside
          // groups of the same size read the same X row (a broadcast) and
          // consecutive Y rows.  Only the lane holding a group's short-to-long
          // switch flushes there; the periodic flushes fall on the same steps in
          // every lane, so a warp runs them together.
          const int P = npairs;                      // pairs (j, d - j), j < d - j
          const bool has_mid = ngroups > P;          // the middle coefficient d/2 pairs with itself
          const int Gp = g_hi - g_lo;                // groups of this part
          int grp = g_hi, q = 0, Q = 1;              // lanes without a group run no terms
          if (Gp > 0) {
            const int Qb = T / Gp;                   // lanes per group (>= 1: the plan sizes T)
            const int extra = T - Qb * Gp;           // the first `extra` groups have Qb + 1 lanes
            if (tid < extra * (Qb + 1)) {
              Q = Qb + 1;
              grp = g_lo + tid / Q;
              q = tid - (grp - g_lo) * Q;
            } else {
              Q = Qb;
              const int t2 = tid - extra * (Qb + 1);
              grp = g_lo + extra + t2 / Q;
              q = t2 - (grp - g_lo - extra) * Q;
            }
          }
          int cs = 0, cl = 0, ns = 0, nl = 0, tp = 0;
          if (grp >= g_hi) {
            // no group: no terms
          } else if (grp < P) {
            cs = conv ? grp : d - grp;               // short coefficient: grp + 1 terms
            cl = conv ? d - grp : grp;               // long coefficient: d - grp + 1 terms
            ns = grp + 1;
            nl = d - grp + 1;
            tp = d + 2;
          } else if (grp == P && has_mid) {
            cs = cl = d / 2;
            ns = d / 2 + 1;
            tp = ns;
          }
          const int H = tp > 0 ? (tp + Q - 1) / Q : 0;
          const int p0 = q * H;
          const int p1 = min(p0 + H, tp);
          int jcur = p0 < ns ? cs : cl;
          int left = R;  // terms the accumulators take before the next flush
          // Exchange rows with one writer each: the lane's private row takes
          // the coefficient it ends on; a lane whose run crosses from the short
          // to the long coefficient puts its short partial sums into its
          // group's extra row.
          unsigned long long* prow = exch + static_cast<size_t>(tid) * private_row_stride(L);
          unsigned long long* cur = prow;
          if (grp < g_hi && p0 < ns && p1 > ns)
            cur = exch + static_cast<size_t>(T + grp - g_lo) * private_row_stride(L);
          for (int pos = p0; pos < p1; ++pos) {
            int j, i;
            if (pos < ns) {
              j = cs;
              i = pos;
            } else {
              j = cl;
              i = nl - 1 - (pos - ns);
            }
            const int ix = conv ? i : j + i;
            const int iy = conv ? j - i : i;
            term(ix, iy, gs[j] - gx[ix] - gy[iy]);
            --left;
            if (pos == ns - 1 && pos + 1 < p1) {
              DigitMac<K, INTV>::flush_own(cur, A);  // this lane leaves the short coefficient
              cur = prow;
              jcur = cl;
            }
            if (left == 0) {  // the same steps in every lane (not reset by the switch)
              DigitMac<K, INTV>::flush_own(cur, A);
              left = R;
            }
          }
          if (p1 > p0) DigitMac<K, INTV>::flush_own(cur, A);
          (void)jcur;
        } else {
          // Every thread runs the same number of consecutive terms of the
          // concatenated term sequence; partial sums of a coefficient split between
          // threads meet exactly in the shared exchange row.
          const long long W = static_cast<long long>(d + 1) * (d + 2) / 2;
          const long long g0 = W * tid / T;
          const long long g1 = W * (tid + 1) / T;
          const int cnt = static_cast<int>(g1 - g0);
          int j = 0, i = 0;
          if (cnt > 0) {
            int lo = 0, hi = d;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              const long long st = conv ? conv_start(mid) : corr_start(mid, d);
              if (st <= g0) lo = mid; else hi = mid - 1;
            }
            j = lo;
            i = static_cast<int>(g0 - (conv ? conv_start(j) : corr_start(j, d)));
          }
          int nt = conv ? j + 1 : d - j + 1;
          int gsj = cnt > 0 ? gs[j] : 0;
          for (int s = 0; s < cnt; ++s) {
            const int ix = conv ? i : j + i;
            const int iy = conv ? j - i : i;
            term(ix, iy, gsj - gx[ix] - gy[iy]);
            ++i;
            const bool end_coef = (i == nt);
            if (end_coef || ((s + 1) % R == 0)) flush(j);
            if (end_coef) {
              ++j;
              i = 0;
              if (j <= d) {
                nt = conv ? j + 1 : d - j + 1;
                gsj = gs[j];
              }
            }
          }
          if (i > 0) flush(j);
        }
      }
      __syncthreads();
      if (ahead && tid == stager) {
        claim();
        stage(false);
      }

      // ---- one output coefficient per thread: the exact sum as L digits on its grid ----
      for (int j = tid; j <= d; j += T) {
        if (!owned(j)) continue;
        const int32_t g = gs[j];
        int32_t o[L];
        int32_t gz = GRID_ZERO;
        if (g < -100000) {
  #pragma unroll
          for (int p = 0; p < L; ++p) o[p] = 0;
        } else {
          int64_t E[L + 1];
          if constexpr (INTV) {
            // the lanes of the coefficient's group that ran its terms: those of
            // the short coefficient before the crossing lane, plus the extra row
            // when a lane crosses; those of the long one from the crossing lane
            // on; every lane for the middle coefficient
            const int grp = min(j, d - j);
            const int r = grp - g_lo, Gp = g_hi - g_lo;
            const int Qb = T / Gp, extra = T - Qb * Gp;
            const int Q = r < extra ? Qb + 1 : Qb;
            const int l0 = r < extra ? r * (Qb + 1) : extra * (Qb + 1) + (r - extra) * Qb;
            const bool mid = (d % 2 == 0) && j == d / 2;
            const int tp = mid ? d / 2 + 1 : d + 2;
            const int ns = mid ? tp : grp + 1;
            const int H = (tp + Q - 1) / Q;
            const int qb = ns / H;
            const bool is_short = !mid && j == (jb.kind == JOB_CONV ? grp : d - grp);
            const int lo = mid ? 0 : is_short ? 0 : qb;
            const int hi = mid ? Q : is_short ? qb : Q;
            constexpr int PS = private_row_stride(L);
#pragma unroll
            for (int t = 0; t <= L; ++t) E[t] = 0;
#pragma unroll 1
            for (int u = l0 + lo; u < l0 + hi; ++u) {
              const long long* row = reinterpret_cast<const long long*>(exch) + static_cast<size_t>(u) * PS;
#pragma unroll
              for (int t = 0; t <= L; ++t) E[t] += row[t];
            }
            if (is_short && ns % H != 0) {
              const long long* row = reinterpret_cast<const long long*>(exch) + static_cast<size_t>(T + r) * PS;
#pragma unroll
              for (int t = 0; t <= L; ++t) E[t] += row[t];
            }
          } else {
#pragma unroll
            for (int t = 0; t <= L; ++t) E[t] = exch_word(exch + j * (L + 1), t);
          }
          gz = sum_to_digits<L, B>(E, g, o);
        }
        int4* dst = reinterpret_cast<int4*>(zrows + static_cast<long long>(j) * RW);
  #pragma unroll
        for (int v = 0; v < RW / 4; ++v)
          dst[v] = make_int4(4 * v < L ? o[4 * v] : 0, 4 * v + 1 < L ? o[4 * v + 1] : 0,
                             4 * v + 2 < L ? o[4 * v + 2] : 0, 4 * v + 3 < L ? o[4 * v + 3] : 0);
        zgrid[j] = gz;
      }
    }
    __syncthreads();
    if (tid == 0) publish_flag(a.flags + sj, epoch);
    claimed = ahead;
  }
}

// ---------------------------------------------------------------------------
// tiled convolution kernel (degrees whose whole series do not fit in shared
// memory)
// ---------------------------------------------------------------------------

// Shared-memory layout of the tiled kernel for tiles of D coefficients: the
// exchange rows of the output tile; the X rows of one tile of the first
// operand and the window of 2D + 4 rows of the second operand they meet; the
// grids of those rows and the reference grid of every output coefficient.
struct TileLayout {
  size_t exch, raw, xdig, ydig, gx, gy, gs, bar, misc, total;
};

__host__ __device__ constexpr int tile_window(int D) { return 2 * D + 4; }

__host__ __device__ inline TileLayout tile_layout(int L, bool intv, int D) {
  const int digit_bytes = intv ? 4 : 8;
  const int W = tile_window(D);
  TileLayout o;
  size_t off = 0;
  o.exch = off;
  off = align_up(off + size_t(D) * (L + 1) * sizeof(unsigned long long), 128);
  o.raw = off;  // X rows as copied (FP64 variant: then the Y window)
  off = align_up(off + size_t(intv ? D : D + W) * row_words(L, intv) * sizeof(int32_t), 128);
  o.xdig = off;
  off = align_up(off + size_t(D) * x_stride(L, intv) * digit_bytes, 16);
  o.ydig = off;  // integer variant: the Y window lands here as copied
  off = align_up(off + size_t(W) * y_stride(L, intv) * digit_bytes, 16);
  o.gx = off;
  off = align_up(off + size_t(D) * 4, 16);
  o.gy = off;
  off = align_up(off + size_t(W) * 4, 16);
  o.gs = off;
  off = align_up(off + size_t(D) * 4, 16);
  o.bar = off;
  off += 16;
  o.misc = off;
  off += 64;
  o.total = align_up(off, 128);
  return o;
}

// Every job is split into output tiles of D = a.tile coefficients; sub-job
// j * a.split + t computes coefficients [tD, tD + D) of job j (a.split tiles
// per job cover the largest degree).  Output coefficient c_j = sum_i x_i y_{j-i}
// (Eq. eqconvform; the correlation sums x_{j+i} y_i) is accumulated tile pair
// by tile pair: for every tile I of the first operand that meets the output
// tile, its D rows and the window of the second operand's rows they pair with
// are staged by TMA bulk copies, and every term of the pair adds into the
// output tile's exchange rows, which stay in shared memory until the last
// tile pair.  The reference grid of each output coefficient is the largest
// grid of its terms over all tiles, taken before the first tile pair, so that
// the exact sums and the L digits they are cut to are those of the
// whole-series kernel, bit for bit.
template <int K, bool INTV>
__global__ void __launch_bounds__(dag_max_threads(K), INTV ? dag_min_ctas(K) : 1) dag_tiled_kernel(DagArgs a) {
  using M = DigitMac<K, INTV>;
  using DigitT = typename M::DigitT;
  using AccT = typename M::AccT;
  constexpr int B = M::B;
  constexpr int L = M::L;
  constexpr int XS = M::XS;
  constexpr int YS = M::YS;
  constexpr int XOFF = M::XOFF;
  constexpr int RW = row_words(L, INTV);
  constexpr int R = INTV ? static_cast<int>((1LL << (63 - 2 * (B - 1))) / L) : 128 / L;

  extern __shared__ __align__(128) unsigned char smem[];
  const int D = a.tile;
  const TileLayout lay = tile_layout(L, INTV, D);
  unsigned long long* exch = reinterpret_cast<unsigned long long*>(smem + lay.exch);
  int32_t* raw = reinterpret_cast<int32_t*>(smem + lay.raw);
  DigitT* xdig = reinterpret_cast<DigitT*>(smem + lay.xdig);
  DigitT* ydig = reinterpret_cast<DigitT*>(smem + lay.ydig);
  int32_t* gx = reinterpret_cast<int32_t*>(smem + lay.gx);
  int32_t* gy = reinterpret_cast<int32_t*>(smem + lay.gy);
  int32_t* gs = reinterpret_cast<int32_t*>(smem + lay.gs);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + lay.bar);
  int32_t* misc = reinterpret_cast<int32_t*>(smem + lay.misc);

  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const uint32_t bar_addr = smem_u32(bar);
  if (tid == 0) {
    mbar_init(bar_addr, 1);
    fence_mbar_init();
  }
  if constexpr (INTV) {
    for (int t = tid; t < D * XS; t += T) xdig[t] = 0;  // zero prefixes of the X rows
  }
  __syncthreads();
  const int epoch = *reinterpret_cast<volatile int32_t*>(&a.ctrl->epoch);
  uint32_t phase = 0;
  const int tiles = parts(a);
  const int nsub = a.njobs * tiles;

  // bulk copies of rows [c0, c0 + cnt) of a series (digit rows to `rows`, grids
  // to `grid`); cnt and c0 are multiples of 4, so every copy is a multiple of
  // 16 bytes from a 16-byte boundary
  auto copy_rows = [&](const int32_t* series, int S, int c0, int cnt, void* rows, int32_t* grid) {
    bulk_g2s(smem_u32(rows), series + static_cast<long long>(c0) * RW, static_cast<uint32_t>(cnt) * RW * 4u,
             bar_addr);
    bulk_g2s(smem_u32(grid), series + static_cast<long long>(S) * RW + c0, static_cast<uint32_t>(cnt) * 4u,
             bar_addr);
  };
  // bounded wait for the copies of the current stage; false: timed out (the
  // copies in flight are then given their own bounded wait before the exit)
  auto landed = [&]() {
    const bool ok = __syncthreads_and(mbar_wait(bar_addr, phase, a.timeout_ns));
    if (!ok) mbar_wait(bar_addr, phase, a.timeout_ns);
    phase ^= 1u;
    return ok;
  };

  for (;;) {
    if (tid == 0) {
      misc[0] = atomicAdd(&a.ctrl->next[a.counter], 1);
      misc[1] = 0;
    }
    __syncthreads();
    const int sj = misc[0];
    if (sj >= nsub) break;
    const int job = sj / tiles;
    const int tile = sj - job * tiles;
    const ConvJob jb = a.jobs[job];
    const InstInfo in = a.inst[jb.inst];
    const int d = in.d, S = in.S;
    const int j0 = tile * D;
    const int jn = min(D, d + 1 - j0);  // output coefficients of this tile (<= 0: none)
    const bool elementwise = jb.kind == JOB_ADD || jb.kind == JOB_SUB;
    const bool conv = jb.kind == JOB_CONV;
    const int last = d / D;  // last tile of this instance's series
    if (jn > 0) {
      // ---- operands: the tiles this output tile reads ----
      if (tid == 0) {
        const int t_lo = elementwise ? tile : 0;
        const int t_hi = (elementwise || conv) ? tile : last;
        bool ok = true;
        for (int t = t_lo; ok && t <= t_hi; ++t) {
          if (jb.dep1 >= 0) ok = wait_flag(a, jb.dep1 * tiles + t, epoch, job);
          if (ok && jb.dep2 >= 0) ok = wait_flag(a, jb.dep2 * tiles + t, epoch, job);
        }
        misc[1] = ok ? 0 : 1;
        fence_proxy_async_global();
        fence_proxy_async_shared();
      }
      __syncthreads();
      if (misc[1]) break;
      const int32_t* xs = a.ws + in.ws_base + static_cast<long long>(jb.in1) * in.ws_sstride;
      const int32_t* ys = a.ws + in.ws_base + static_cast<long long>(jb.in2) * in.ws_sstride;
      int32_t* zrows = a.ws + in.ws_base + static_cast<long long>(jb.out) * in.ws_sstride;
      int32_t* zgrid = zrows + static_cast<long long>(S) * RW;
      int32_t* ywin = INTV ? reinterpret_cast<int32_t*>(ydig) : raw + D * RW;  // Y rows as copied

      if (elementwise) {
        // ---- out = in1 +- in2 on the rows of this tile, exactly, as L digits ----
        const int cnt = min(D, S - j0);
        if (tid == 0) {
          fence_proxy_async_shared();
          mbar_expect_tx(bar_addr, 2u * static_cast<uint32_t>(cnt) * (RW + 1) * 4u);
          copy_rows(xs, S, j0, cnt, raw, gx);
          copy_rows(ys, S, j0, cnt, ywin, gy);
        }
        if (!landed()) {
          if (tid == 0) set_error(a.ctrl, kStatusTimeout, job, -2);
          break;
        }
        const long long sgn = jb.kind == JOB_SUB ? -1 : 1;
        for (int t = tid; t < jn; t += T) {
          const int32_t g = max(gx[t], gy[t]);
          int32_t o[L];
          int32_t gz = GRID_ZERO;
          if (g < -100000) {
#pragma unroll
            for (int p = 0; p < L; ++p) o[p] = 0;
          } else {
            const int sx = g - gx[t], sy = g - gy[t];
            int64_t E[L + 1];
            E[0] = 0;
#pragma unroll
            for (int q = 0; q < L; ++q) {
              const long long xv = q >= sx ? raw[t * RW + q - sx] : 0;
              const long long yv = q >= sy ? ywin[t * RW + q - sy] : 0;
              E[q + 1] = xv + sgn * yv;
            }
            gz = sum_to_digits<L, B>(E, g + 1, o);
          }
          int4* dst = reinterpret_cast<int4*>(zrows + static_cast<long long>(j0 + t) * RW);
#pragma unroll
          for (int v = 0; v < RW / 4; ++v)
            dst[v] = make_int4(4 * v < L ? o[4 * v] : 0, 4 * v + 1 < L ? o[4 * v + 1] : 0,
                               4 * v + 2 < L ? o[4 * v + 2] : 0, 4 * v + 3 < L ? o[4 * v + 3] : 0);
          zgrid[j0 + t] = gz;
        }
      } else {
        // ---- reference grid of every output coefficient: the largest grid
        // of its terms, a warp per coefficient over the operands' grids ----
        const int32_t* gX = xs + static_cast<long long>(S) * RW;
        const int32_t* gY = ys + static_cast<long long>(S) * RW;
        for (int t = warp; t < D; t += nwarps) {
          const int j = j0 + t;
          int32_t m = 2 * GRID_ZERO;
          if (t < jn) {
            const int n = conv ? j + 1 : d - j + 1;
            for (int i = lane; i < n; i += 32)
              m = max(m, conv ? __ldcg(gX + i) + __ldcg(gY + j - i) : __ldcg(gX + j + i) + __ldcg(gY + i));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0) gs[t] = m;
        }
        for (int t = tid; t < D * (L + 1); t += T) exch[t] = 0ull;

        // Lanes: the output tile's coefficients a = j0 + g and b = j0 + D-1-g
        // form group g (D/2 groups); each group gets T / (D/2) consecutive lanes
        // (the first T mod (D/2) groups one more), which split the group's terms
        // of the tile pair in consecutive runs.  In a full tile pair every
        // coefficient has D terms; in the diagonal one a and b have D + 1
        // together.  One of the two is walked forwards and the other backwards,
        // so that lanes of the same rank read the same X row in every group (a
        // broadcast) and consecutive Y rows.  (Taking the terms in turn instead,
        // lane q the terms q, q + Q, ..., avoids the bank conflicts between
        // ranks D/Q rows apart but measured 3 % slower.)
        const int G = D / 2;
        const int Qb = T / G, extra = T - Qb * G;
        int grp, q, Q;
        if (tid < extra * (Qb + 1)) {
          Q = Qb + 1;
          grp = tid / Q;
          q = tid - grp * Q;
        } else {
          Q = Qb;
          const int t2 = tid - extra * (Qb + 1);
          grp = extra + t2 / Q;
          q = t2 - (grp - extra) * Q;
        }
        const int ca = j0 + grp, cb = j0 + D - 1 - grp;  // the group's two coefficients
        const int i_first = conv ? 0 : tile, i_last = conv ? tile : last;
        bool ok = true;
        for (int I = i_first; I <= i_last; ++I) {
          const int i0 = I * D;
          // first-operand index range of every coefficient of the tile pair
          auto range = [&](int j, int& lo, int& hi) {
            if (j > d) {
              lo = hi = 0;
            } else if (conv) {
              lo = i0;
              hi = min(i0 + D, j + 1);
            } else {
              lo = max(i0, j);
              hi = min(i0 + D, d + 1);
            }
            if (hi < lo) hi = lo;
          };
          // second-operand window: conv j - i, corr i - j, over the tile pair
          const int ymin = conv ? j0 - (i0 + D - 1) : i0 - (j0 + jn - 1);
          const int ymax = min(d, conv ? j0 + jn - 1 - i0 : i0 + D - 1 - j0);
          const int y0 = max(0, ymin) & ~3;
          const int ycnt = min((ymax - y0 + 1 + 3) & ~3, S - y0);
          const int xcnt = min(D, S - i0);
          __syncthreads();  // the previous tile pair's rows are no longer read
          if (tid == 0) {
            fence_proxy_async_shared();
            mbar_expect_tx(bar_addr, static_cast<uint32_t>(xcnt + ycnt) * (RW + 1) * 4u);
            copy_rows(xs, S, i0, xcnt, raw, gx);
            copy_rows(ys, S, y0, ycnt, ywin, gy);
          }
          if (!landed()) {
            if (tid == 0) set_error(a.ctrl, kStatusTimeout, job, -2);
            ok = false;
            break;
          }
          // ---- staged digit rows into the layouts of the multiply-accumulate loop ----
          if constexpr (INTV) {
            constexpr int V4 = RW / 4;
            const int4* src = reinterpret_cast<const int4*>(raw);
            for (int t = tid; t < xcnt * V4; t += T) {
              const int c = t / V4, v = t - c * V4;
              const int4 qv = src[t];
              int32_t* dst = xdig + c * XS + XOFF + 4 * v;
              if (4 * v < L) dst[0] = qv.x;
              if (4 * v + 1 < L) dst[1] = qv.y;
              if (4 * v + 2 < L) dst[2] = qv.z;
              if (4 * v + 3 < L) dst[3] = qv.w;
            }
          } else {
            for (int t = tid; t < xcnt * L; t += T) {
              const int c = t / L, p = t - c * L;
              xdig[c * XS + p] = static_cast<double>(raw[c * RW + p]);
            }
            for (int t = tid; t < ycnt * L; t += T) {
              const int c = t / L, p = t - c * L;
              ydig[c * YS + p] = static_cast<double>(ywin[c * RW + p]);
            }
          }
          __syncthreads();

          // ---- multiply-accumulate the group's terms of this tile pair ----
          int lo_a, hi_a, lo_b, hi_b;
          range(ca, lo_a, hi_a);
          range(cb, lo_b, hi_b);
          const int na = hi_a - lo_a, tp = na + (hi_b - lo_b);
          const int H = (tp + Q - 1) / Q;
          const int p0 = min(q * H, tp), p1 = min(p0 + H, tp);
          AccT A[L];
#pragma unroll
          for (int t = 0; t < L; ++t) acc_clear(A[t]);
          int jcur = p0 < na ? ca : cb;
          int left = R;
          for (int pos = p0; pos < p1; ++pos) {
            int j, x;
            if (pos < na) {
              j = ca;
              x = conv ? lo_a + pos : hi_a - 1 - pos;
            } else {
              j = cb;
              x = conv ? hi_b - 1 - (pos - na) : lo_b + (pos - na);
            }
            const int iy = conv ? j - x : x - j;
            const int lx = x - i0, ly = iy - y0;
            M::term(xdig, ydig, lx, ly, gs[j - j0] - gx[lx] - gy[ly], A);
            --left;
            if (pos == na - 1 && pos + 1 < p1) {
              M::flush(exch + (ca - j0) * (L + 1), A);  // this lane leaves coefficient a
              jcur = cb;
            }
            if (left == 0) {  // the same steps in every lane
              M::flush(exch + (jcur - j0) * (L + 1), A);
              left = R;
            }
          }
          if (p1 > p0) M::flush(exch + (jcur - j0) * (L + 1), A);
        }
        if (!ok) break;
        __syncthreads();

        // ---- one output coefficient per thread: the exact sum as L digits on its grid ----
        for (int t = tid; t < jn; t += T) {
          const int32_t g = gs[t];
          int32_t o[L];
          int32_t gz = GRID_ZERO;
          if (g < -100000) {
#pragma unroll
            for (int p = 0; p < L; ++p) o[p] = 0;
          } else {
            int64_t E[L + 1];
#pragma unroll
            for (int u = 0; u <= L; ++u) E[u] = exch_word(exch + t * (L + 1), u);
            gz = sum_to_digits<L, B>(E, g, o);
          }
          int4* dst = reinterpret_cast<int4*>(zrows + static_cast<long long>(j0 + t) * RW);
#pragma unroll
          for (int v = 0; v < RW / 4; ++v)
            dst[v] = make_int4(4 * v < L ? o[4 * v] : 0, 4 * v + 1 < L ? o[4 * v + 1] : 0,
                               4 * v + 2 < L ? o[4 * v + 2] : 0, 4 * v + 3 < L ? o[4 * v + 3] : 0);
          zgrid[j0 + t] = gz;
        }
      }
    }
    __syncthreads();
    if (tid == 0) publish_flag(a.flags + sj, epoch);
  }
}

// ---------------------------------------------------------------------------
// pack / unpack
// ---------------------------------------------------------------------------

// pack: one warp per series; every lane converts coefficients j = lane, lane+32,
// ... of the caller's k-limb series into L balanced digits on the grid of the
// leading limb and writes the digit row and grid into the workspace slot.
template <int K, bool INTV>
__global__ void __launch_bounds__(256) pack_kernel(CopyArgs a) {
  constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  constexpr int L = digits_for_k(K, B);
  constexpr int RW = row_words(L, INTV);
  const long long row = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= a.nrows) return;
  const CopyRow r = a.rows[row];
  const InstInfo in = a.inst[r.inst];
  const double* src = a.src[r.sel] + r.off;
  int32_t* rows = a.ws + in.ws_base + static_cast<long long>(r.slot) * in.ws_sstride;
  int32_t* grids = rows + static_cast<long long>(in.S) * RW;
  for (int j = lane; j <= in.d; j += 32) {
    int64_t D[L];
    const int32_t g = grid_of<B>(src[j]);
    to_digits<K, L, B>(src + j, r.lstride, g, D);
    int4* dst = reinterpret_cast<int4*>(rows + static_cast<long long>(j) * RW);
#pragma unroll
    for (int v = 0; v < RW / 4; ++v)
      dst[v] = make_int4(4 * v < L ? static_cast<int32_t>(D[4 * v]) : 0,
                         4 * v + 1 < L ? static_cast<int32_t>(D[4 * v + 1]) : 0,
                         4 * v + 2 < L ? static_cast<int32_t>(D[4 * v + 2]) : 0,
                         4 * v + 3 < L ? static_cast<int32_t>(D[4 * v + 3]) : 0);
    grids[j] = g;
  }
}

// unpack: one warp per series; every lane rounds coefficients of a workspace
// series (digit form) to k limbs in the caller's buffer.
template <int K, bool INTV>
__global__ void __launch_bounds__(256) unpack_kernel(CopyArgs a) {
  constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  constexpr int L = digits_for_k(K, B);
  constexpr int RW = row_words(L, INTV);
  const long long row = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= a.nrows) return;
  const CopyRow r = a.rows[row];
  const InstInfo in = a.inst[r.inst];
  double* dst = a.dst[r.sel] + r.off;
  const int32_t* rows = a.ws + in.ws_base + static_cast<long long>(r.slot) * in.ws_sstride;
  const int32_t* grids = rows + static_cast<long long>(in.S) * RW;
  for (int j = lane; j <= in.d; j += 32) {
    const int32_t g = grids[j];
    if (g < -100000) {
#pragma unroll
      for (int l = 0; l < K; ++l) dst[l * r.lstride + j] = 0.0;
      continue;
    }
    int64_t E[L + 1];
    E[0] = 0;
#pragma unroll
    for (int p = 0; p < L; ++p) E[p + 1] = rows[static_cast<long long>(j) * RW + p];
    from_digits<K, L, B>(E, g + 1, dst + j, r.lstride);
  }
}

__global__ void prologue_kernel(Ctrl* ctrl) {
  if (threadIdx.x == 0) {
    ctrl->epoch += 1;
#pragma unroll
    for (int c = 0; c < 4; ++c) ctrl->next[c] = 0;
  }
}

// ---------------------------------------------------------------------------
// addition stage: warp per output coefficient, exact digit sums, warp shuffles
// ---------------------------------------------------------------------------

// GROUPED: group_warps warps per output coefficient (block barriers combine
// them); else one warp per output coefficient and no barrier.
template <int K, bool INTV, bool GROUPED>
__device__ __forceinline__ void add_body(const AddArgs& a, long long items, long long blk) {
  constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  constexpr int L = digits_for_k(K, B);
  constexpr int RW = row_words(L, INTV);
  // a group of group_warps warps per output coefficient (outputs with many
  // contributions spread them over more lanes); every thread reaches the
  // block barriers, so lanes past the last item only skip the work
  __shared__ int32_t gm_s[8];
  __shared__ long long acc_s[8][L];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = GROUPED ? a.group_warps : 1;
  const int G = gw * 32;
  const int sw = warp % gw;                  // warp within the group
  const int gl = sw * 32 + lane;             // lane within the group
  const long long w = blk * (8 / gw) + warp / gw;
  const bool valid = w < items;
  AddOut ao{};
  int j = 0;
  InstInfo in{};
  if (valid) {
    int lo = 0, hi = a.nouts - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.item_ptr[mid] <= w) lo = mid; else hi = mid - 1;
    }
    ao = a.outs[lo];
    j = static_cast<int>(w - a.item_ptr[lo]);
    in = a.inst[ao.inst];
  }
  const int32_t* base = a.ws + in.ws_base;
  const long long gofs = static_cast<long long>(in.S) * RW + j;  // grid of coefficient j within a slot
  const long long rofs = static_cast<long long>(j) * RW;         // row of coefficient j within a slot

  // item index of a real single plan (value: output 0, d p / d x_i: output 1 + i)
  const long long item =
      (ao.dst_sel == 0 ? 0 : 1 + ao.dst_off / (in.d + 1)) * static_cast<long long>(in.d + 1) + j;

  // common grid: the largest grid of the contributions (mode 2: the one given)
  int32_t gmax = 2 * GRID_ZERO;
  if (a.mode == 2) {
    gmax = valid ? a.grid_io[item] : gmax;
  } else {
    if (valid) {
#pragma unroll 4
      for (int c = ao.cbeg + gl; c < ao.cend; c += G)
        gmax = max(gmax, base[static_cast<long long>(a.contrib[c]) * in.ws_sstride + gofs]);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if constexpr (GROUPED) {
      if (lane == 0) gm_s[warp] = gmax;
      __syncthreads();
      for (int t = 0; t < gw; ++t) gmax = max(gmax, gm_s[warp - sw + t]);
    }
    if (a.mode == 1) {
      if (valid && gl == 0) a.grid_io[item] = gmax;
      return;  // (every thread has passed the group's barrier)
    }
  }

  // every lane sums its contributions' digits, shifted to the common grid
  int64_t acc[L];
#pragma unroll
  for (int p = 0; p < L; ++p) acc[p] = 0;
  if (valid && gmax >= -100000) {
#pragma unroll 2
    for (int c = ao.cbeg + gl; c < ao.cend; c += G) {
      const int32_t* slot = base + static_cast<long long>(a.contrib[c]) * in.ws_sstride;
      const int sh = gmax - slot[gofs];  // digits below the common grid's top
      if (sh >= L) continue;               // below the last digit
      const int32_t* row = slot + rofs;
      const long long mu = a.mult ? a.mult[c] : 1;  // the exponent of the variable (Sec. 3)
#pragma unroll
      for (int q = 0; q < L; ++q)
        if (q >= sh) acc[q] += mu * row[q - sh];
    }
  }
#pragma unroll
  for (int p = 0; p < L; ++p) {
    long long v = acc[p];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[p] = v;
  }
  if constexpr (GROUPED) {
    if (lane == 0)
#pragma unroll
      for (int p = 0; p < L; ++p) acc_s[warp][p] = acc[p];
    __syncthreads();
    if (sw == 0 && lane == 0)
      for (int t = 1; t < gw; ++t)
#pragma unroll
        for (int p = 0; p < L; ++p) acc[p] += acc_s[warp + t][p];
  }
  if (!valid || gl != 0) return;
  if (a.mode == 2) {
#pragma unroll
    for (int p = 0; p < L; ++p) a.acc_out[item * L + p] = acc[p];
    return;
  }
  // acc[p] weighs 2^(B (gmax - 1 - p)): word p + 1 of a sum on grid gmax + 1
  int64_t E[L + 1];
  E[0] = 0;
#pragma unroll
  for (int p = 0; p < L; ++p) E[p + 1] = acc[p];
  if (a.to_ws) {
    int32_t* slot = a.ws + in.ws_base + ao.dst_off * in.ws_sstride;
    int32_t o[L];
    const int32_t gz = gmax < -100000 ? GRID_ZERO : sum_to_digits<L, B>(E, gmax + 1, o);
    if (gmax < -100000) {
#pragma unroll
      for (int p = 0; p < L; ++p) o[p] = 0;
    }
    int4* dst = reinterpret_cast<int4*>(slot + rofs);
#pragma unroll
    for (int v = 0; v < RW / 4; ++v)
      dst[v] = make_int4(4 * v < L ? o[4 * v] : 0, 4 * v + 1 < L ? o[4 * v + 1] : 0,
                         4 * v + 2 < L ? o[4 * v + 2] : 0, 4 * v + 3 < L ? o[4 * v + 3] : 0);
    slot[gofs] = gz;
    return;
  }
  double* dst = a.dst[ao.dst_sel] + ao.dst_off + j * ao.dst_jstride;
  if (gmax < -100000) {
#pragma unroll
    for (int l = 0; l < K; ++l) dst[l * ao.dst_lstride] = 0.0;
    return;
  }
  from_digits<K, L, B>(E, gmax + 1, dst, ao.dst_lstride);
}

template <int K, bool INTV>
__global__ void __launch_bounds__(256) add_kernel(AddArgs a, long long items) {
  add_body<K, INTV, false>(a, items, blockIdx.x);
}

// Digit sums on their grids (acc[p] weighs 2^(B (g - 1 - p)), g = grids[item])
// rounded to k limbs, as the addition stage rounds its own sums: item
// o (d + 1) + j is coefficient j of the value (o = 0) or of d p / d x_{o-1}.
template <int K, bool INTV>
__host__ __device__ void round_sum_item(const RoundArgs& a, long long item) {
  constexpr int B = INTV ? DIGIT_BITS_INT : DIGIT_BITS;
  constexpr int L = digits_for_k(K, B);
  const long long D1 = a.d + 1;
  const long long o = item / D1, j = item - o * D1;
  double* dst = o == 0 ? a.value + j : a.grad + (o - 1) * D1 + j;
  const long long ls = o == 0 ? D1 : static_cast<long long>(a.n) * D1;
  const int32_t g = a.grids[item];
  if (g < -100000) {
    for (int l = 0; l < K; ++l) dst[l * ls] = 0.0;
    return;
  }
  int64_t E[L + 1];
  E[0] = 0;
  for (int p = 0; p < L; ++p) E[p + 1] = a.acc[item * L + p];
  from_digits<K, L, B>(E, g + 1, dst, ls);
}

template <int K, bool INTV>
__global__ void __launch_bounds__(256) round_sums_kernel(RoundArgs a, long long items) {
  const long long item = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (item < items) round_sum_item<K, INTV>(a, item);
}

template <int K, bool INTV>
void round_sums_host_k(const RoundArgs& a) {
  const long long items = static_cast<long long>(a.n + 1) * (a.d + 1);
  for (long long item = 0; item < items; ++item) round_sum_item<K, INTV>(a, item);
}

template <int K, bool INTV>
__global__ void __launch_bounds__(256) add_kernel_grouped(AddArgs a, long long items) {
  add_body<K, INTV, true>(a, items, blockIdx.x);
}

// Both parts of an addition stage whose outputs are all summed by groups of
// warps, in one launch: the first nb0 blocks take part 0, the rest part 1 (the
// branch is uniform over a block, so the group barriers hold).
template <int K, bool INTV>
__global__ void __launch_bounds__(256) add_kernel_pair(AddArgs a0, long long items0, AddArgs a1, long long items1,
                                                       unsigned nb0) {
  if (blockIdx.x < nb0)
    add_body<K, INTV, true>(a0, items0, blockIdx.x);
  else
    add_body<K, INTV, true>(a1, items1, blockIdx.x - nb0);
}

// ---------------------------------------------------------------------------
// elementwise multiple double operations
// ---------------------------------------------------------------------------

template <int K>
__global__ void md_binary_kernel(int op, const double* x, const double* y, double* out, long long count) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double a[K], b[K], r[K];
#pragma unroll
  for (int l = 0; l < K; ++l) {
    a[l] = x[l * count + i];
    b[l] = y[l * count + i];
  }
  if (op == 0)
    md::md_add<K>(a, b, r);
  else
    md::md_mul<K>(a, b, r);
#pragma unroll
  for (int l = 0; l < K; ++l) out[l * count + i] = r[l];
}

// DFMA throughput: 8 independent FMA chains per thread.
__global__ void fp64_peak_kernel(double* sink, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = __fma_rn(acc[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  if (s == 12345.678) sink[blockIdx.x] = s;  // keeps the chains alive
}

// 32x32->64 multiply-add throughput in the form the convolution kernel issues:
// 64-bit accumulators and multiplicands read from shared memory.  Every
// iteration loads two rows of 8 digits (the row index changes with the
// iteration, so the compiler cannot hoist the products out of the loop; with
// constant operands it turns the loop into 64-bit additions, which run on
// another pipe) and accumulates their 8 x 8 outer product into 8 accumulators.
__global__ void __launch_bounds__(256) int_peak_kernel(long long* sink, int iters, int a, int b) {
  __shared__ __align__(16) int32_t rows[64 * 8];
  for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) rows[t] = static_cast<int32_t>((t * 2654435761u) & 0x7FFFFFF) - a;
  __syncthreads();
  long long acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 7LL * threadIdx.x + i + b;
  for (int it = 0; it < iters; ++it) {
    const int4* p = reinterpret_cast<const int4*>(rows + ((it + threadIdx.x) & 63) * 8);
    const int4* q = reinterpret_cast<const int4*>(rows + ((7 * it + threadIdx.x) & 63) * 8);
    const int4 u = p[0], v = p[1], w = q[0], z = q[1];
    const int X[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
    const int Y[8] = {w.x, w.y, w.z, w.w, z.x, z.y, z.z, z.w};
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[i]) : "r"(X[i]), "r"(Y[j]));
  }
  long long s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  if (s == 12345) sink[blockIdx.x] = s;
}

// The kernel a launch uses: the tiled kernel, the narrow whole-series
// instantiation (k <= 2, integer pipe, at most kNarrowThreads threads) or the
// general one.
template <int K, bool INTV>
void* dag_fn(bool tiled, bool narrow) {
  if (tiled) return reinterpret_cast<void*>(&dag_tiled_kernel<K, INTV>);
  if constexpr (dag_has_narrow(K, INTV)) {
    if (narrow) return reinterpret_cast<void*>(&dag_kernel<K, INTV, true>);
  }
  return reinterpret_cast<void*>(&dag_kernel<K, INTV>);
}

void* dag_kernel_ptr(int k, int arith, bool tiled, bool narrow) {
  const bool iv = arith == ARITH_INT;
  switch (k) {
    case 1: return iv ? dag_fn<1, true>(tiled, narrow) : dag_fn<1, false>(tiled, narrow);
    case 2: return iv ? dag_fn<2, true>(tiled, narrow) : dag_fn<2, false>(tiled, narrow);
    case 3: return iv ? dag_fn<3, true>(tiled, narrow) : dag_fn<3, false>(tiled, narrow);
    case 4: return iv ? dag_fn<4, true>(tiled, narrow) : dag_fn<4, false>(tiled, narrow);
    case 5: return iv ? dag_fn<5, true>(tiled, narrow) : dag_fn<5, false>(tiled, narrow);
    case 8: return iv ? dag_fn<8, true>(tiled, narrow) : dag_fn<8, false>(tiled, narrow);
    case 10: return iv ? dag_fn<10, true>(tiled, narrow) : dag_fn<10, false>(tiled, narrow);
    default: return nullptr;
  }
}

bool narrow_launch(int threads) { return threads > 0 && threads <= kNarrowThreads; }

}  // namespace

int digits_of_k(int k, int arith) { return digits_for_k(k, arith == ARITH_INT ? DIGIT_BITS_INT : DIGIT_BITS); }

int ws_row_words(int k, int arith) { return row_words(digits_of_k(k, arith), arith == ARITH_INT); }

size_t dag_smem_bytes(int k, int arith, int smax, int dmax, int depth, int threads) {
  return dag_layout(k, digits_of_k(k, arith), arith == ARITH_INT, smax, dmax, depth, threads).total;
}

size_t dag_tiled_smem_bytes(int k, int arith, int tile) {
  return tile_layout(digits_of_k(k, arith), arith == ARITH_INT, tile).total;
}

// The dynamic shared-memory limit is a property of the kernel function on a
// device, shared by every plan: raise it, never lower it, so that a plan built
// later for a smaller degree cannot break the launches of an earlier one.
cudaError_t dag_prepare(int k, int arith, size_t smem, bool tiled) {
  void* fn = dag_kernel_ptr(k, arith, tiled, false);
  void* fn_narrow = dag_kernel_ptr(k, arith, tiled, true);  // the same kernel unless k <= 2 whole-series integer
  if (!fn || !fn_narrow) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, bool>, size_t> granted;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = granted[std::make_tuple(dev, k, arith, tiled)];
  if (smem <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e == cudaSuccess && fn_narrow != fn)
    e = cudaFuncSetAttribute(fn_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e == cudaSuccess) cur = smem;
  return e;
}

cudaError_t dag_occupancy(int k, int arith, int threads, size_t smem, int* blocks_per_sm, bool tiled) {
  void* fn = dag_kernel_ptr(k, arith, tiled, narrow_launch(threads));
  if (!fn) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t launch_dag(const DagArgs& a, int k, int arith, int threads, int grid, cudaStream_t st) {
  const bool tiled = a.tile > 0;
  void* fn = dag_kernel_ptr(k, arith, tiled, narrow_launch(threads));
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem =
      tiled ? dag_tiled_smem_bytes(k, arith, a.tile) : dag_smem_bytes(k, arith, a.smax, a.dmax, a.depth, threads);
  DagArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st);
}

cudaError_t launch_prologue(Ctrl* ctrl, cudaStream_t st) {
  prologue_kernel<<<1, 32, 0, st>>>(ctrl);
  return cudaGetLastError();
}

// Launch KERNEL<K, INTV><<<grid, block, 0, st>>>(args...) for run-time k and arith.
#define PES_DISPATCH_K_ARITH(KERNEL, k, arith, grid, block, st, ...)                        \
  do {                                                                                      \
    const bool iv_ = (arith) == ARITH_INT;                                                  \
    switch (k) {                                                                            \
      case 1: if (iv_) KERNEL<1, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<1, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 2: if (iv_) KERNEL<2, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<2, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 3: if (iv_) KERNEL<3, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<3, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 4: if (iv_) KERNEL<4, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<4, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 5: if (iv_) KERNEL<5, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<5, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 8: if (iv_) KERNEL<8, true><<<grid, block, 0, st>>>(__VA_ARGS__);                 \
              else KERNEL<8, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;             \
      case 10: if (iv_) KERNEL<10, true><<<grid, block, 0, st>>>(__VA_ARGS__);               \
               else KERNEL<10, false><<<grid, block, 0, st>>>(__VA_ARGS__); break;           \
      default: return cudaErrorInvalidValue;                                                \
    }                                                                                       \
  } while (0)

cudaError_t launch_pack(const CopyArgs& a, int k, int arith, cudaStream_t st) {
  if (a.nrows == 0) return cudaSuccess;
  const int warps = 8;
  const unsigned grid = static_cast<unsigned>((a.nrows + warps - 1) / warps);
  PES_DISPATCH_K_ARITH(pack_kernel, k, arith, grid, warps * 32, st, a);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const CopyArgs& a, int k, int arith, cudaStream_t st) {
  if (a.nrows == 0) return cudaSuccess;
  const int warps = 8;
  const unsigned grid = static_cast<unsigned>((a.nrows + warps - 1) / warps);
  PES_DISPATCH_K_ARITH(unpack_kernel, k, arith, grid, warps * 32, st, a);
  return cudaGetLastError();
}

cudaError_t launch_add(const AddArgs& a, int k, int arith, int64_t items, cudaStream_t st) {
  if (items == 0) return cudaSuccess;
  if (!(a.group_warps == 1 || a.group_warps == 2 || a.group_warps == 4 || a.group_warps == 8))
    return cudaErrorInvalidValue;
  const int warps = 8;
  const int per_block = warps / a.group_warps;  // output coefficients per block
  const unsigned grid = static_cast<unsigned>((items + per_block - 1) / per_block);
  if (a.group_warps > 1)
    PES_DISPATCH_K_ARITH(add_kernel_grouped, k, arith, grid, warps * 32, st, a, static_cast<long long>(items));
  else
    PES_DISPATCH_K_ARITH(add_kernel, k, arith, grid, warps * 32, st, a, static_cast<long long>(items));
  return cudaGetLastError();
}

cudaError_t launch_add_pair(const AddArgs& a0, int64_t items0, const AddArgs& a1, int64_t items1, int k,
                            int arith, cudaStream_t st) {
  const auto grouped = [](int gw) { return gw == 2 || gw == 4 || gw == 8; };
  if (!grouped(a0.group_warps) || !grouped(a1.group_warps)) return cudaErrorInvalidValue;
  const int warps = 8;
  const long long pb0 = warps / a0.group_warps, pb1 = warps / a1.group_warps;
  const unsigned nb0 = static_cast<unsigned>((items0 + pb0 - 1) / pb0);
  const unsigned grid = nb0 + static_cast<unsigned>((items1 + pb1 - 1) / pb1);
  PES_DISPATCH_K_ARITH(add_kernel_pair, k, arith, grid, warps * 32, st, a0, static_cast<long long>(items0), a1,
                       static_cast<long long>(items1), nb0);
  return cudaGetLastError();
}

cudaError_t launch_round_sums(const RoundArgs& a, int k, int arith, cudaStream_t st) {
  const long long items = static_cast<long long>(a.n + 1) * (a.d + 1);
  if (items == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((items + 255) / 256);
  PES_DISPATCH_K_ARITH(round_sums_kernel, k, arith, grid, 256, st, a, items);
  return cudaGetLastError();
}

int round_sums_host(int k, int arith, const RoundArgs& a) {
  const bool iv = arith == ARITH_INT;
  switch (k) {
    case 1: iv ? round_sums_host_k<1, true>(a) : round_sums_host_k<1, false>(a); return 0;
    case 2: iv ? round_sums_host_k<2, true>(a) : round_sums_host_k<2, false>(a); return 0;
    case 3: iv ? round_sums_host_k<3, true>(a) : round_sums_host_k<3, false>(a); return 0;
    case 4: iv ? round_sums_host_k<4, true>(a) : round_sums_host_k<4, false>(a); return 0;
    case 5: iv ? round_sums_host_k<5, true>(a) : round_sums_host_k<5, false>(a); return 0;
    case 8: iv ? round_sums_host_k<8, true>(a) : round_sums_host_k<8, false>(a); return 0;
    case 10: iv ? round_sums_host_k<10, true>(a) : round_sums_host_k<10, false>(a); return 0;
    default: return 1;
  }
}

cudaError_t launch_md_binary(int op, int k, const double* x, const double* y, double* out, int64_t count,
                             cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((count + 127) / 128);
  switch (k) {
    case 1: md_binary_kernel<1><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 2: md_binary_kernel<2><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 3: md_binary_kernel<3><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 4: md_binary_kernel<4><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 5: md_binary_kernel<5><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 8: md_binary_kernel<8><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    case 10: md_binary_kernel<10><<<grid, 128, 0, st>>>(op, x, y, out, count); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_int_peak(long long* sink, int blocks, int threads, int iters, cudaStream_t st) {
  int_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters, 3, 5);
  return cudaGetLastError();
}

cudaError_t launch_fp64_peak(double* sink, int blocks, int threads, int iters, cudaStream_t st) {
  fp64_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters, 0.999999999, 1e-9);
  return cudaGetLastError();
}

}  // namespace pes
