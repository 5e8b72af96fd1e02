// Host build of the library's digit arithmetic (csrc/digits.cuh), for CPU tests
// of the exact dot product against the oracle.  Test code only: it mirrors the
// arithmetic of the convolution and addition kernels one coefficient at a time.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../paper_2101_10881_gb300/csrc/digits.cuh"

using namespace pes;

namespace {

template <int K, int B>
void conv_k(int d, const double* x, const double* y, double* z, int corr) {
  constexpr int L = digits_for_k(K, B);
  const int S = d + 1;
  std::vector<int32_t> gx(S), gy(S);
  std::vector<int64_t> X(static_cast<size_t>(S) * L), Y(static_cast<size_t>(S) * L);
  for (int c = 0; c < S; ++c) {
    int64_t D[L];
    gx[c] = grid_of<B>(x[c]);
    to_digits<K, L, B>(x + c, S, gx[c], D);
    for (int p = 0; p < L; ++p) X[c * L + p] = D[p];
    gy[c] = grid_of<B>(y[c]);
    to_digits<K, L, B>(y + c, S, gy[c], D);
    for (int p = 0; p < L; ++p) Y[c * L + p] = D[p];
  }
  for (int j = 0; j <= d; ++j) {
    const int nt = corr ? d - j + 1 : j + 1;
    int32_t gs = 2 * GRID_ZERO;
    for (int i = 0; i < nt; ++i) {
      int ix = corr ? j + i : i, iy = corr ? i : j - i;
      gs = std::max(gs, gx[ix] + gy[iy]);
    }
    if (gs < -100000) {
      for (int l = 0; l < K; ++l) z[l * S + j] = 0.0;
      continue;
    }
    int64_t E[L + 1] = {0};
    for (int i = 0; i < nt; ++i) {
      int ix = corr ? j + i : i, iy = corr ? i : j - i;
      int delta = gs - gx[ix] - gy[iy];
      if (delta >= L) continue;
      for (int p = 0; p < L; ++p) {
        int id = p - delta;
        int64_t xv = id < 0 ? 0 : X[ix * L + id];
        for (int q = 0; q < L - p; ++q) E[p + q + 1] += xv * Y[iy * L + q];
      }
    }
    from_digits<K, L, B>(E, gs, z + j, S);
  }
}

template <int K>
void sum_k(int count, const double* v, double* out) {
  constexpr int L = digits_for_k(K);
  int32_t g = 2 * GRID_ZERO;
  for (int c = 0; c < count; ++c) g = std::max(g, grid_of(v[c]));
  if (g < -100000) {
    for (int l = 0; l < K; ++l) out[l] = 0.0;
    return;
  }
  int64_t E[L + 1] = {0};
  for (int c = 0; c < count; ++c) {
    int64_t D[L];
    to_digits<K, L>(v + c, count, g, D);
    for (int p = 0; p < L; ++p) E[p] += D[p];
  }
  from_digits<K, L>(E, g, out, 1);
}

}  // namespace

#define DISPATCH(k, call)     \
  switch (k) {                \
    case 1: call(1); break;   \
    case 2: call(2); break;   \
    case 3: call(3); break;   \
    case 4: call(4); break;   \
    case 5: call(5); break;   \
    case 8: call(8); break;   \
    case 10: call(10); break; \
    default: return 1;        \
  }

extern "C" int hd_conv(int k, int d, const double* x, const double* y, double* z, int corr, int bits) {
  if (bits == 24) {
#define C(K) conv_k<K, 24>(d, x, y, z, corr)
    DISPATCH(k, C)
#undef C
  } else if (bits == 28) {
#define C(K) conv_k<K, 28>(d, x, y, z, corr)
    DISPATCH(k, C)
#undef C
  } else {
    return 1;
  }
  return 0;
}

// v: limb-major [k][count]; out: k limbs of the sum
extern "C" int hd_sum(int k, int count, const double* v, double* out) {
#define C(K) sum_k<K>(count, v, out)
  DISPATCH(k, C)
#undef C
  return 0;
}

extern "C" int hd_digits(int k) {
  int r = 0;
#define C(K) r = digits_for_k(K)
  DISPATCH(k, C)
#undef C
  return r;
}
