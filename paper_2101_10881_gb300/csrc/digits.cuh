// digits.cuh -- exact fixed-point digits for multiple double dot products.
//
// A k-double number x (limbs x[0..k-1], nonoverlapping, |x[0]| largest) is
// written on a grid g (an integer) as
//     x ~= 2^(B g) * sum_{p=0..L-1} X_p 2^(-B (p+1)),   |X_p| <= 2^(B-1),
// with B-bit balanced digits X_p.  With B = 24, products of two digits are at
// most 2^46 in magnitude, exact in a double, and sums of up to 128 of them stay
// exact in a double (2^53); with B = 28 products are below 2^54 and sums of 512
// of them stay exact in an int64.  That is what makes the multiply-accumulate
// loop of a truncated series product (Eq. eqconvform) an error-free
// transformation: every term x_i y_{j-i} is accumulated exactly into digit
// positions, and the sum is rounded once to k limbs at the end.
//
// The number of digits L per k is chosen so that the dropped tail of every term
// is below 2^-(53k+12) of the largest term (see digits_for_k).
//
// All conversions (limbs -> digits, digits -> limbs) use integer operations only;
// the FP64 pipe is left to the multiply-accumulate loop.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define PES_HD __host__ __device__ __forceinline__
#define PES_HDC __host__ __device__ constexpr
#else
#define PES_HD inline
#define PES_HDC constexpr
#endif

namespace pes {

PES_HD uint64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
#endif
}

PES_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll(static_cast<long long>(x));
#else
  return __builtin_clzll(x);
#endif
}

// Digit width B: 24 bits for FP64 accumulation (digit products below 2^46, sums
// of 128 of them exact in a double), 28 bits for 64-bit integer accumulation
// (products below 2^54, sums of 512 of them exact in an int64).
constexpr int DIGIT_BITS = 24;
constexpr int DIGIT_BITS_INT = 28;
// grid of a zero coefficient: far below any real grid so that every term with
// it is skipped
constexpr int32_t GRID_ZERO = -(1 << 28);

// L: smallest number of digits with B (L - 1) >= 53 k + 28 (12 guard bits plus
// log2 of (1024 terms x 40 digit products)), see the error budget above.
PES_HDC int digits_for_k(int k, int B = DIGIT_BITS) { return (53 * k + 28 + B - 1) / B + 1; }

PES_HD int32_t floordiv(int32_t a, int32_t b) {
  int32_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Decode a double into sign, 53-bit integer mantissa and exponent of its lsb:
// x = sign * mant * 2^lsb.  Returns false for zero.
PES_HD bool decode(double x, int& neg, uint64_t& mant, int32_t& lsb) {
  uint64_t bits = dbits(x);
  uint32_t be = static_cast<uint32_t>((bits >> 52) & 0x7FF);
  uint64_t frac = bits & ((uint64_t(1) << 52) - 1);
  neg = static_cast<int>(bits >> 63);
  if (be == 0) {
    if (frac == 0) return false;
    mant = frac;
    lsb = -1074;
  } else {
    mant = frac | (uint64_t(1) << 52);
    lsb = static_cast<int32_t>(be) - 1075;
  }
  return true;
}

// Grid of a k-double whose leading limb is x0: g = ceil((e + 2) / B) where
// |x| <= 2^e, so that |x| <= 2^(B g - 2).
template <int B = DIGIT_BITS>
PES_HD int32_t grid_of(double x0) {
  uint64_t bits = dbits(x0);
  uint32_t be = static_cast<uint32_t>((bits >> 52) & 0x7FF);
  if ((bits << 1) == 0) return GRID_ZERO;
  int32_t e = (be == 0 ? 1 : static_cast<int32_t>(be)) - 1022;  // |x0| < 2^e
  return floordiv(e + 2 + B - 1, B);
}

// Signed piece of limb (neg, mant, lsb) inside the digit window whose lsb is at
// absolute bit position P (bits [P, P + B)), truncated toward zero.
template <int B>
PES_HD int64_t window(int neg, uint64_t mant, int32_t lsb, int32_t P) {
  int32_t sh = P - lsb;
  uint64_t v;
  if (sh >= 0)
    v = sh >= 64 ? 0 : (mant >> sh);
  else
    v = (-sh) >= B ? 0 : (mant << (-sh));
  int64_t piece = static_cast<int64_t>(v & ((uint64_t(1) << B) - 1));
  return neg ? -piece : piece;
}

// Digits of a k-double on grid g into D[0..L-1], balanced.  x: limb l at
// x[l * ls].  Each limb's 53 bits fall into at most four consecutive digit
// windows, so only those are touched (D is indexed at run time).  Bits below the
// last digit are dropped.
template <int K, int L, int B = DIGIT_BITS>
PES_HD void to_digits(const double* x, long long ls, int32_t g, int64_t (&D)[L]) {
#pragma unroll
  for (int p = 0; p < L; ++p) D[p] = 0;
  const int32_t top = B * g;  // bit position just above digit 0
#pragma unroll 1
  for (int l = 0; l < K; ++l) {
    int neg;
    uint64_t mant;
    int32_t lsb;
    if (!decode(x[l * ls], neg, mant, lsb)) continue;
    const int32_t hb = lsb + 52;  // highest bit of the limb (mantissas of normal numbers)
    int32_t p0 = floordiv(top - 1 - hb, B);
    if (p0 < 0) p0 = 0;
    if (p0 >= L) break;  // this limb and every smaller one lie below the last digit
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int p = p0 + r;
      if (p < L) D[p] += window<B>(neg, mant, lsb, top - B * (p + 1));
    }
  }
  // balanced digits: carry from the bottom up
#pragma unroll
  for (int p = L - 1; p >= 1; --p) {
    int64_t c = (D[p] + (int64_t(1) << (B - 1))) >> B;
    D[p] -= c << B;
    D[p - 1] += c;
  }
}

// The exact sum V = sum_{a=0..L} E[a] 2^(B (gs - 1 - a)) as L balanced digits
// on a grid of its own: returns that grid g' and out[0..L-1] (digit p weighs
// 2^(B (g' - 1 - p))), the top digit nonzero; GRID_ZERO and zero digits when
// V = 0.  The digits are carried from the bottom into [-2^(B-1), 2^(B-1)), the
// top word spills into up to two more digits above it (any 64-bit word fits),
// leading zero digits are shifted out (a barrel shift over fixed indices, so
// everything stays in registers), and the digits below the L kept ones are
// dropped: being balanced, they weigh at most about half a unit of the last
// kept digit.
template <int L, int B>
PES_HD int32_t sum_to_digits(int64_t (&E)[L + 1], int32_t gs, int32_t (&out)[L]) {
  constexpr int64_t HALF = int64_t(1) << (B - 1);
  constexpr int N = L + 3;  // F[0], F[1]: digits above E[0]; F[a + 2] = E[a]
#pragma unroll
  for (int a = L; a >= 1; --a) {
    const int64_t c = (E[a] + HALF) >> B;
    E[a] -= c << B;
    E[a - 1] += c;
  }
  int64_t F[N];
  {
    const int64_t c1 = (E[0] + HALF) >> B;
    const int64_t c2 = (c1 + HALF) >> B;
    F[0] = c2;
    F[1] = c1 - (c2 << B);
    F[2] = E[0] - (c1 << B);
  }
#pragma unroll
  for (int a = 1; a <= L; ++a) F[a + 2] = E[a];
  int z = N;  // index of the first nonzero digit
#pragma unroll
  for (int i = N - 1; i >= 0; --i)
    if (F[i] != 0) z = i;
  if (z == N) {
#pragma unroll
    for (int p = 0; p < L; ++p) out[p] = 0;
    return GRID_ZERO;
  }
#pragma unroll
  for (int b = 1; b < N; b <<= 1) {
    if (z & b) {
#pragma unroll
      for (int i = 0; i < N; ++i) F[i] = (i + b < N) ? F[i + b] : 0;
    }
  }
#pragma unroll
  for (int p = 0; p < L; ++p) out[p] = static_cast<int32_t>(F[p]);
  // F[z] sat at a = z - 2, weighing 2^(B (gs + 1 - z)) = 2^(B (g' - 1))
  return gs + 2 - z;
}

// Round the exact fixed-point sum V = sum_{a=0..L} E[a] 2^(B (L - a)) times
// 2^(B gs - B (L + 1)) to K nonoverlapping limbs (each limb the nearest double
// to the remainder, ties away from zero), written to out[l * ls].
//
// The digits are first carried into [0, 2^B) (digit 0 keeps the sign), then the
// magnitude is packed into 64-bit words; each limb takes the 53 bits below the
// highest set bit, rounded; the remainder is V with those bits cleared, or, when
// the limb was rounded up, 2^mexp minus the bits below mexp with the sign flipped.
template <int K, int L, int B = DIGIT_BITS>
PES_HD void from_digits(int64_t (&E)[L + 1], int32_t gs, double* out, long long ls) {
  constexpr int NA = L + 1;
  constexpr int NW = (B * L + 64 + 63) / 64 + 1;  // digit 0 holds < 2^44
  auto normalise = [&]() {
#pragma unroll
    for (int a = NA - 1; a >= 1; --a) {
      int64_t c = E[a] >> B;
      E[a] -= c << B;
      E[a - 1] += c;
    }
  };
  normalise();
  double sign = 1.0;
  if (E[0] < 0) {
#pragma unroll
    for (int a = 0; a < NA; ++a) E[a] = -E[a];
    normalise();
    sign = -1.0;
  }
  // pack: digit a occupies bits [B (L - a), B (L - a) + B) (digit 0: upwards)
  uint64_t Wd[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) Wd[w] = 0;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int pos = B * (L - a);
    const int w = pos / 64, o = pos % 64;
    const uint64_t v = static_cast<uint64_t>(E[a]);
    Wd[w] |= v << o;
    if (o > 0 && w + 1 < NW) Wd[w + 1] |= v >> (64 - o);
  }
  const int32_t base_exp = B * gs - B * (L + 1);
#pragma unroll 1
  for (int l = 0; l < K; ++l) {
    int tw = -1;
#pragma unroll
    for (int w = 0; w < NW; ++w)
      if (Wd[w] != 0) tw = w;
    if (tw < 0) {
      for (int r = l; r < K; ++r) out[r * ls] = 0.0;
      return;
    }
    uint64_t hi = 0, lo = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      if (w == tw) hi = Wd[w];
      if (w == tw - 1) lo = Wd[w];
    }
    const int hb = 63 - clz64(hi);          // top bit inside word tw
    const int32_t h = 64 * tw + hb;         // top bit of V
    // W = the 64 bits of V whose highest is bit h
    const uint64_t W = (hb == 63) ? hi : ((hi << (63 - hb)) | (lo >> (hb + 1)));
    const uint64_t rbit = (W >> 10) & 1;
    const uint64_t m = (W >> 11) + rbit;    // 53 bits, rounded to nearest
    const int32_t mexp = h - 52;            // weight of the mantissa lsb (may be negative)
    out[l * ls] = sign * ldexp(static_cast<double>(m), mexp + base_exp);
    if (mexp <= 0) {
      // every bit of V was taken (exactly, rounding adds nothing below bit 0)
      for (int r = l + 1; r < K; ++r) out[r * ls] = 0.0;
      return;
    }
    const int wm = mexp / 64, om = mexp % 64;
    if (!rbit) {
      // remainder: V with bits >= mexp cleared
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        if (w > wm) Wd[w] = 0;
        if (w == wm) Wd[w] &= (om == 0) ? 0 : ((uint64_t(1) << om) - 1);
      }
    } else {
      // remainder: -(2^mexp - (V mod 2^mexp)); keep the magnitude, flip the sign
      uint64_t borrow = 1;  // two's complement of the bits below mexp: ~x + 1
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        if (w < wm) {
          const uint64_t nv = ~Wd[w] + borrow;
          borrow = (borrow && nv == 0) ? 1 : 0;
          Wd[w] = nv;
        } else if (w == wm) {
          const uint64_t mask = (om == 0) ? 0 : ((uint64_t(1) << om) - 1);
          Wd[w] = (~Wd[w] + borrow) & mask;
        } else {
          Wd[w] = 0;
        }
      }
      sign = -sign;
    }
  }
}

}  // namespace pes
