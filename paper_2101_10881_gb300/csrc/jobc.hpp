// jobc.hpp -- host job-table compiler (integer only, no CUDA).
//
// Turns monomial supports into the convolution jobs of the reverse mode of
// Sec. 3 (forward products f, backward products b, cross products c) placed in
// layers (Sec. 5, "Jobs are placed in layers"), and into the addition work of
// the second stage (Sec. 5, pairs of the tree summation).  The same tables drive
// one polynomial or a batch of them: a batch is the concatenation of the
// instances' tables, each instance with its own workspace region and degree.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace pes {

// Job kinds.
// CONV: out = in1 * in2 truncated (Eq. eqconvform); CORR: the truncated
// correlation of the VJP; ADD / SUB: out = in1 + in2 / in1 - in2, coefficient
// by coefficient (complex products combine their real products with them).
enum : int32_t { JOB_CONV = 0, JOB_CORR = 1, JOB_ADD = 2, JOB_SUB = 3 };

// Where instance `inst` keeps series slot s (in int32 words from the workspace
// base): slot s starts at ws_base + s * ws_sstride and holds S rows of digits
// (coefficient j at row j, a fixed number of words per row), then the S grids.
struct InstInfo {
  int64_t ws_base;
  int64_t ws_sstride;
  int32_t S;  // padded series length (multiple of 8 coefficients)
  int32_t d;  // truncation degree
};

// One convolution (or correlation) job: out := in1 * in2 (slots of one instance).
// dep1/dep2: index of the job that produces in1/in2 in the same job list, or -1
// when the operand is an input series.
struct ConvJob {
  int32_t in1, in2, out;
  int32_t dep1, dep2;
  int32_t inst;
  int32_t kind;
  int32_t layer;
};

// One output series of the addition stage: the exact sum of the series in
// contrib[cbeg, cend) (slots of instance `inst`), rounded to k limbs and
// written to destination buffer `dst_sel` at dst_off + l * dst_lstride + j, or,
// for an addition into the workspace, kept in digit form in slot dst_off.
struct AddOut {
  int64_t dst_off;
  int64_t dst_lstride;
  int32_t dst_sel;
  int32_t inst;
  int32_t cbeg, cend;
  int64_t dst_jstride = 1;  // distance between coefficients j and j+1 in the destination
};

// One series copy between a caller buffer and the workspace.  For a pack (caller
// to workspace) src is the caller buffer `sel`; for an unpack it is the target.
struct CopyRow {
  int64_t off;      // caller-buffer offset of coefficient 0, limb 0 (doubles)
  int64_t lstride;  // caller-buffer limb stride (doubles)
  int32_t sel;      // which caller buffer
  int32_t inst;
  int32_t slot;     // workspace slot
  int32_t pad;
};

// Slots of one monomial in the product layout.
struct MonoSlots {
  int32_t nk;
  int32_t f0;   // f_{k,1}..f_{k,nk}: f0 .. f0+nk-1
  int32_t b0;   // b_{k,1}..: b0 ..
  int32_t nb;   // number of b slots (max(1, nk-2) for nk>=2, 0 for nk==1)
  int32_t bA;   // slot of b_{k,nk-2} * a_k (nk >= 3), else -1
  int32_t c0;   // c_{k,1}..c_{k,nk-2}
  int32_t nc;
};

// Parsed, validated supports of one polynomial.
struct Supports {
  int32_t N = 0, n = 0;
  std::vector<int32_t> ptr, idx;  // CSR, 0-based, increasing per row
  std::vector<int32_t> ex;        // exponent of every support entry (empty: all 1)
  int32_t exponent(int32_t t) const { return ex.empty() ? 1 : ex[static_cast<size_t>(t)]; }
};

// Largest exponent a monomial may give one variable.
constexpr int32_t kMaxExponent = 64;

// Returns "" if valid, else a message.  Rules: N >= 0, n >= 1, every monomial
// non-empty, indices in [0, n), strictly increasing within a monomial.
std::string validate(const int32_t* ptr, const int32_t* idx, int32_t N, int32_t n);
// Exponents (one per support entry): "" if every one lies in [1, kMaxExponent].
std::string validate_exponents(const int32_t* ptr, const int32_t* ex, int32_t N);

// Layout and jobs of one polynomial (slot numbering local to the instance).
struct Program1 {
  int32_t N = 0, n = 0, d = 0;
  int32_t n_input_slots = 0;   // 1 + N + n (a_0, a_1..a_N, z_1..z_n)
  int32_t n_slots = 0;         // total slots of the eval+grad layout
  int32_t n_layers = 0;
  std::vector<MonoSlots> mono;
  std::vector<ConvJob> jobs;   // sorted by layer (stable in monomial order)
  std::vector<int32_t> layer_ptr;      // jobs of layer L (1-based) at [layer_ptr[L-1], layer_ptr[L])
  // addition stage: output 0 = value, output 1+i = d p / d x_i
  std::vector<int32_t> add_ptr;        // n+2 entries
  std::vector<int32_t> add_src;        // contributing slots
  std::vector<int32_t> add_mult;       // integer factor of every contribution (the exponent of the variable)
  // per monomial: its terms of the addition stage, (output, slot, factor) with
  // output 0 the value and 1 + i the partial for x_i
  std::vector<std::vector<std::array<int32_t, 3>>> mono_terms;
  // systems (compile_system): P polynomials, constant term of polynomial p in slot const0 + p;
  // with VJP tables: upstream series u_p in slot_up0 + p, the Jacobian series in digit form
  // in slot_J0 + p*n + i, their correlations with u_p in slot_rJ0 + p*n + i
  int32_t system_P = 0, const0 = -1;
  int32_t slot_up0 = -1, slot_J0 = -1, slot_rJ0 = -1;
  // monomials with powers (Sec. 3): series powers z_v^q, common factors and the
  // coefficients a'_m = a_m * prod z_v^(e_v - 1) that the reverse mode uses
  bool has_powers = false;
  int32_t power_jobs = 0;              // jobs of the power table, the common factors and the a'_m
  // VJP extras (slots after the eval+grad layout)
  int32_t slot_u = -1;                 // upstream series
  int32_t slot_M0 = -1;                // M_k (k = 1..N) at slot_M0 + k - 1 (or an input slot, see mslot)
  std::vector<int32_t> mslot;          // slot holding M_k (input slot when nk == 1)
  int32_t slot_g0 = -1;                // gradient series g_i at slot_g0 + i
  int32_t slot_r0 = -1;                // correlation outputs: N coefficient + n input series
  int32_t n_slots_vjp = 0;
  std::vector<ConvJob> vjp_jobs;       // forward jobs + M jobs (topological), then correlation jobs
  int32_t vjp_fwd_jobs = 0;            // number of conv jobs before the correlations
  std::vector<ConvJob> vjp_mjobs;      // the M jobs alone (for a VJP that reuses the forward products)
};

// Build the eval+grad layout and jobs.  paper_layout=true reproduces the data
// array of Eq. (eqcountnum) (b_{k,nk-2} updated in place, no VJP extras); it is
// used for the offset/count checks against the paper only.
Program1 compile(const Supports& s, int32_t d, bool paper_layout = false, bool with_vjp = false);

// A system of P polynomials in the same n variables (Newton's method on series
// evaluates one): monomials poly_ptr[p] .. poly_ptr[p+1]-1 of s belong to
// polynomial p.  The products are those of compile(s, d); the addition stage
// has P value outputs (the constant term of polynomial p in slot const0 + p,
// then its monomials) followed by the P x n Jacobian entries, output
// P + p * n + i = d p_p / d x_i.  With VJP tables (for L = sum_p <u_p, v_p>):
// the forward products and the monomial products M_m of compile(s, d, false,
// true), then the correlations of u_p with M_m (slot_r0 + m, m in polynomial p)
// and with every nonempty Jacobian series (slot_rJ0 + p*n + i); the gradient
// for x_i is the sum over p of the latter.
Program1 compile_system(const Supports& s, const std::vector<int32_t>& poly_ptr, int32_t d, bool with_vjp = false);

// The same polynomial over complex series: every slot s of the real program
// becomes the pair (2s, 2s + 1) (real, imaginary part), every product
// x * y becomes four real products xr yr, xi yi, xr yi, xi yr (four scratch
// slots) and the ADD / SUB jobs re = xr yr - xi yi, im = xr yi + xi yr; the
// addition stage sums real and imaginary parts separately, output 2o the real
// and 2o + 1 the imaginary part of output o of the real program.  With VJP
// tables in `real`, its correlations of u with s become correlations with
// conj(s) (the gradient of the real loss sum Re u Re v + Im u Im v with
// respect to real and imaginary parts); the VJP slot fields keep their
// real-layout numbers.  Every job sits in the earliest layer its operands allow.
Program1 complexify(const Program1& real);

// Addition-tree level sizes of the paper's pairwise summation (Sec. 5, read with
// a_0 as one more term of the value sum): each level pairs floor(m/2) of a list
// of m terms, for the value and for every gradient sum.
std::vector<int64_t> paper_add_levels(const Supports& s);

// Padded series stride for degree d (multiple of 8 doubles, 64 bytes).
inline int32_t series_stride(int32_t d) { return ((d + 1) + 7) / 8 * 8; }

}  // namespace pes
