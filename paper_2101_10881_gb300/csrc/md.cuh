// md.cuh -- multiple double arithmetic on the device (k = 1,2,3,4,5,8,10 limbs).
//
// Numbers are unevaluated sums of K doubles with nonoverlapping limbs of
// decreasing magnitude (Sec. 1, multiple double arithmetic).  Operations are
// built from the FMA-based error-free transformations:
//   TwoSum      s + e == a + b       (6 flops, any order of a, b)
//   FastTwoSum  s + e == a + b       (3 flops, |a| >= |b|)
//   TwoProd     p + e == a * b       (2 flops with one FMA)
// and a renormalisation (a VecSum pass from the bottom, then a top-down pass
// that emits nonzero errors as the next limb).
//
// md_add and md_mul are the paper's two operations on numbers.  The series
// kernels do not call them term by term: they use the exact digit dot product of
// digits.cuh, which rounds a whole convolution coefficient once.
#pragma once

namespace pes {
namespace md {

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

// N roughly magnitude-ordered terms -> K nonoverlapping limbs.
template <int N, int K>
__device__ __forceinline__ void renorm(double (&v)[N], double (&r)[K]) {
  // VecSum from the bottom: v[0] becomes the rounded sum, v[1..] exact errors
#pragma unroll
  for (int i = N - 1; i >= 1; --i) two_sum(v[i - 1], v[i], v[i - 1], v[i]);
#pragma unroll
  for (int q = 0; q < K; ++q) r[q] = 0.0;
  int j = 0;
  double eps = v[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    double s, e;
    fast_two_sum(eps, v[i], s, e);
    if (e != 0.0) {
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (q == j) r[q] = s;
      ++j;
      eps = e;
    } else {
      eps = s;
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == j) r[q] = eps;
}

// out = a + b
template <int K>
__device__ void md_add(const double (&a)[K], const double (&b)[K], double (&out)[K]) {
  // merge by decreasing magnitude (both inputs are normalised)
  double v[2 * K];
  int ia = 0, ib = 0;
  for (int t = 0; t < 2 * K; ++t) {
    bool take_a;
    if (ia >= K)
      take_a = false;
    else if (ib >= K)
      take_a = true;
    else
      take_a = fabs(a[ia]) >= fabs(b[ib]);
    v[t] = take_a ? a[ia++] : b[ib++];
  }
  renorm<2 * K, K>(v, out);
}

// acc[s..K-1] += x with the rounding error of every level carried down; the
// last slot acc[K] collects what is below K limbs.
template <int K>
__device__ __forceinline__ void deposit(double (&acc)[K + 1], int s, double x) {
#pragma unroll
  for (int t = 0; t < K; ++t)
    if (t >= s) two_sum(acc[t], x, acc[t], x);
  acc[K] = __dadd_rn(acc[K], x);
}

// out = a * b, truncated: limb products of order p + q <= K - 1, with the
// TwoProd errors of orders <= K - 2 carried to the next order.
template <int K>
__device__ void md_mul(const double (&a)[K], const double (&b)[K], double (&out)[K]) {
  double acc[K + 1];
#pragma unroll
  for (int t = 0; t <= K; ++t) acc[t] = 0.0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
#pragma unroll
    for (int p = 0; p <= s; ++p) {
      const int q = s - p;
      if (s < K - 1) {
        double h, l;
        two_prod(a[p], b[q], h, l);
        deposit<K>(acc, s, h);
        deposit<K>(acc, s + 1, l);
      } else {
        deposit<K>(acc, K - 1, __dmul_rn(a[p], b[q]));
      }
    }
  }
  renorm<K + 1, K>(acc, out);
}

}  // namespace md
}  // namespace pes
