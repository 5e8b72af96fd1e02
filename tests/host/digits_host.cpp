// Host build of the library's digit arithmetic (csrc/digits.cuh), for CPU tests
// of the exact dot product against the oracle.  Test code only: it mirrors the
// arithmetic of the convolution and addition kernels one coefficient at a time.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../paper_2101_10881_gb300/csrc/digits.cuh"

using namespace pes;

namespace {

// The exact digit sums of one convolution / correlation: grids gs[j] and the
// L+1 words E[j][0..L] (E[a] weighs 2^(B (gs - 1 - a))), as the kernel's
// exchange rows hold them after all flushes.
template <int K, int B>
void conv_words(int d, const double* x, const double* y, int corr, std::vector<int32_t>& gsv,
                std::vector<int64_t>& words) {
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
  gsv.assign(S, 0);
  words.assign(static_cast<size_t>(S) * (L + 1), 0);
  for (int j = 0; j <= d; ++j) {
    const int nt = corr ? d - j + 1 : j + 1;
    int32_t gs = 2 * GRID_ZERO;
    for (int i = 0; i < nt; ++i) {
      int ix = corr ? j + i : i, iy = corr ? i : j - i;
      gs = std::max(gs, gx[ix] + gy[iy]);
    }
    gsv[j] = gs;
    if (gs < -100000) continue;
    int64_t* E = &words[static_cast<size_t>(j) * (L + 1)];
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
  }
}

// Convolution whose result stays in digit form (the kernels' workspace form),
// then rounded to k limbs as the unpack and addition kernels do: digits o on
// grid g are the words (0, o[0..L-1]) on grid g + 1.
template <int K, int B>
void conv_via_digits_k(int d, const double* x, const double* y, double* z, int corr) {
  constexpr int L = digits_for_k(K, B);
  const int S = d + 1;
  std::vector<int32_t> gsv;
  std::vector<int64_t> words;
  conv_words<K, B>(d, x, y, corr, gsv, words);
  for (int j = 0; j <= d; ++j) {
    int64_t E[L + 1];
    for (int a = 0; a <= L; ++a) E[a] = words[static_cast<size_t>(j) * (L + 1) + a];
    int32_t o[L];
    const int32_t g = gsv[j] < -100000 ? GRID_ZERO : sum_to_digits<L, B>(E, gsv[j], o);
    if (g < -100000) {
      for (int l = 0; l < K; ++l) z[l * S + j] = 0.0;
      continue;
    }
    int64_t F[L + 1];
    F[0] = 0;
    for (int p = 0; p < L; ++p) F[p + 1] = o[p];
    from_digits<K, L, B>(F, g + 1, z + j, S);
  }
}

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

extern "C" int hd_conv_via_digits(int k, int d, const double* x, const double* y, double* z, int corr, int bits) {
  if (bits == 24) {
#define C(K) conv_via_digits_k<K, 24>(d, x, y, z, corr)
    DISPATCH(k, C)
#undef C
  } else if (bits == 28) {
#define C(K) conv_via_digits_k<K, 28>(d, x, y, z, corr)
    DISPATCH(k, C)
#undef C
  } else {
    return 1;
  }
  return 0;
}

// sum_to_digits on caller words: E[0..L] (L = digits of k at `bits`), grid gs;
// writes L digits to out and returns the new grid.
template <int K, int B>
int32_t s2d_k(const int64_t* E, int32_t gs, int32_t* out) {
  constexpr int L = digits_for_k(K, B);
  int64_t W[L + 1];
  for (int a = 0; a <= L; ++a) W[a] = E[a];
  int32_t o[L];
  const int32_t g = sum_to_digits<L, B>(W, gs, o);
  for (int p = 0; p < L; ++p) out[p] = o[p];
  return g;
}

extern "C" int hd_sum_to_digits(int k, int bits, const int64_t* E, int32_t gs, int32_t* out, int32_t* grid) {
  if (bits == 24) {
#define C(K) *grid = s2d_k<K, 24>(E, gs, out)
    DISPATCH(k, C)
#undef C
  } else if (bits == 28) {
#define C(K) *grid = s2d_k<K, 28>(E, gs, out)
    DISPATCH(k, C)
#undef C
  } else {
    return 1;
  }
  return 0;
}

extern "C" int hd_digits_bits(int k, int bits) {
  int r = 0;
#define C(K) r = digits_for_k(K, bits)
  DISPATCH(k, C)
#undef C
  return r;
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
