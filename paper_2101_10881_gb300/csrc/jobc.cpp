// jobc.cpp -- host job-table compiler.  See jobc.hpp.
//
// Reverse mode of one monomial a x_{i_1} ... x_{i_n} (Sec. 3), with the index
// readings that the paper's own counts confirm:
//   f_1 = a * z_{i_1},  f_l = f_{l-1} * z_{i_l}                (layer l)
//   b_1 = z_{i_n} * z_{i_{n-1}},  b_l = b_{l-1} * z_{i_{n-l}}   (layer l, l <= n-2)
//   bA  = b_{n-2} * a                                          (layer n-1)
//   c_j = f_j * b_{n-2-j}, j = 1..n-3        (layer max(j, n-2-j) + 1)
//   c_{n-2} = f_{n-2} * z_{i_n}                                (layer n-1)
// giving 3n-3 products; the value term is f_n and the partials are
//   d/dx_{i_1} = bA, d/dx_{i_{j+1}} = c_j (j = 1..n-2), d/dx_{i_n} = f_{n-1}.
// Small monomials (the paper assumes n > 2): n = 2 uses f_1, f_2 and
// b_1 = z_{i_2} * a (3 products); n = 1 uses f_1 = a * z_{i_1} and its partial
// is the coefficient series a itself.
// bA is kept in its own slot (the paper updates b_{n-2} in place) so that the
// product of the variables alone stays available to the VJP.
//
// Monomials with positive powers (Sec. 3): a x_{i_1}^{e_1} ... x_{i_n}^{e_n} is
// a' x_{i_1} ... x_{i_n} with the common factor F = prod z_{i_v}^{e_v - 1}
// folded into the coefficient, a' = a * F, which the reverse mode above then
// uses in place of a.  The powers z^q come from a table built by repeated
// products (z^2 = z z, z^q = z^{q-1} z), F is the product of the powers its
// variables need, and the partial for x_{i_v} is e_v times the exponent-one
// partial (the derivative of z^{e} is e z^{e-1}): the addition stage adds that
// contribution with the integer factor e_v.  Every job sits in the earliest
// layer its operands allow.
#include "jobc.hpp"

#include <algorithm>
#include <numeric>

namespace pes {

std::string validate(const int32_t* ptr, const int32_t* idx, int32_t N, int32_t n) {
  if (N < 0) return "N must be >= 0";
  if (n < 1) return "n must be >= 1";
  if (N > 0 && (ptr == nullptr || idx == nullptr)) return "null support arrays";
  if (N > 0 && ptr[0] != 0) return "supp_ptr[0] must be 0";
  for (int32_t m = 0; m < N; ++m) {
    if (ptr[m + 1] <= ptr[m]) return "empty or decreasing monomial row " + std::to_string(m);
    for (int32_t t = ptr[m]; t < ptr[m + 1]; ++t) {
      if (idx[t] < 0 || idx[t] >= n) return "variable index out of range in monomial " + std::to_string(m);
      if (t > ptr[m] && idx[t] <= idx[t - 1])
        return "indices not strictly increasing in monomial " + std::to_string(m);
    }
  }
  return "";
}

std::string validate_exponents(const int32_t* ptr, const int32_t* ex, int32_t N) {
  if (ex == nullptr) return "";
  for (int32_t t = 0; t < (N > 0 ? ptr[N] : 0); ++t)
    if (ex[t] < 1 || ex[t] > kMaxExponent)
      return "exponent out of [1, " + std::to_string(kMaxExponent) + "] at support entry " + std::to_string(t);
  return "";
}

namespace {

struct Builder {
  std::vector<ConvJob> jobs;
  void add(int32_t in1, int32_t in2, int32_t out, int32_t layer, int32_t kind = JOB_CONV) {
    jobs.push_back(ConvJob{in1, in2, out, -1, -1, 0, kind, layer});
  }
};

// Stable sort by layer, then resolve producer jobs of every operand slot.
// Within a layer, the jobs whose output another job reads come first, so that
// the dependency chains advance as early as the dispatch order allows and the
// leaves (products only the addition stage reads) fill in behind them.
void finalize(std::vector<ConvJob>& jobs, int32_t n_slots) {
  std::vector<char> read(static_cast<size_t>(n_slots), 0);
  for (const ConvJob& j : jobs) {
    read[static_cast<size_t>(j.in1)] = 1;
    read[static_cast<size_t>(j.in2)] = 1;
  }
  std::stable_sort(jobs.begin(), jobs.end(), [&read](const ConvJob& a, const ConvJob& b) {
    if (a.layer != b.layer) return a.layer < b.layer;
    return read[static_cast<size_t>(a.out)] > read[static_cast<size_t>(b.out)];
  });
  std::vector<int32_t> producer(static_cast<size_t>(n_slots), -1);
  for (size_t j = 0; j < jobs.size(); ++j) {
    ConvJob& jb = jobs[j];
    jb.dep1 = producer[static_cast<size_t>(jb.in1)];
    jb.dep2 = producer[static_cast<size_t>(jb.in2)];
    producer[static_cast<size_t>(jb.out)] = static_cast<int32_t>(j);
  }
}

}  // namespace

Program1 compile(const Supports& s, int32_t d, bool paper_layout, bool with_vjp) {
  Program1 P;
  P.N = s.N;
  P.n = s.n;
  P.d = d;
  const int32_t N = s.N, n = s.n;
  auto A = [](int32_t k) { return k; };                 // coefficient a_k, k = 1..N
  auto Z = [N](int32_t v) { return 1 + N + v; };         // input z_v, v 0-based
  P.n_input_slots = 1 + N + n;

  // ---- slot layout (Eq. eqcountnum order: inputs, all f, all b, all c) ----
  P.mono.resize(static_cast<size_t>(N));
  int32_t next = P.n_input_slots;
  for (int32_t m = 0; m < N; ++m) {
    MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    ms.nk = s.ptr[m + 1] - s.ptr[m];
    ms.f0 = next;
    next += ms.nk;
  }
  for (int32_t m = 0; m < N; ++m) {
    MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    ms.nb = paper_layout ? std::max(1, ms.nk - 2) : (ms.nk >= 2 ? std::max(1, ms.nk - 2) : 0);
    ms.b0 = next;
    next += ms.nb;
  }
  for (int32_t m = 0; m < N; ++m) {
    MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    ms.nc = std::max(0, ms.nk - 2);
    ms.c0 = next;
    next += ms.nc;
  }
  for (int32_t m = 0; m < N; ++m) {
    MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    if (ms.nk >= 3) {
      if (paper_layout) {
        ms.bA = ms.b0 + ms.nk - 3;  // in place: b_{k,nk-2}
      } else {
        ms.bA = next++;
      }
    } else {
      ms.bA = -1;
    }
  }
  P.n_slots = next;

  // ---- power table, common factors and a' (monomials with exponents > 1) ----
  // q-th power of z_v: the input slot for q = 1, else a table slot
  std::vector<int32_t> qmax(static_cast<size_t>(n), 1);
  for (int32_t t = 0; t < (N > 0 ? s.ptr[static_cast<size_t>(N)] : 0); ++t)
    qmax[static_cast<size_t>(s.idx[static_cast<size_t>(t)])] =
        std::max(qmax[static_cast<size_t>(s.idx[static_cast<size_t>(t)])], s.exponent(t) - 1);
  std::vector<int32_t> pow0(static_cast<size_t>(n), -1);  // slot of z_v^2 (z_v^q at pow0 + q - 2)
  for (int32_t v = 0; v < n; ++v) {
    if (qmax[static_cast<size_t>(v)] >= 2) {
      pow0[static_cast<size_t>(v)] = next;
      next += qmax[static_cast<size_t>(v)] - 1;
      P.has_powers = true;
    }
  }
  auto POW = [&](int32_t v, int32_t q) { return q == 1 ? Z(v) : pow0[static_cast<size_t>(v)] + q - 2; };
  std::vector<int32_t> acoef(static_cast<size_t>(N));  // slot of the coefficient the reverse mode uses
  std::vector<std::vector<int32_t>> fchain(static_cast<size_t>(N));  // common-factor chain slots
  for (int32_t m = 0; m < N; ++m) {
    acoef[static_cast<size_t>(m)] = A(m + 1);
    int32_t np = 0;
    for (int32_t t = s.ptr[static_cast<size_t>(m)]; t < s.ptr[static_cast<size_t>(m) + 1]; ++t)
      np += s.exponent(t) >= 2;
    if (np == 0) continue;
    P.has_powers = true;
    for (int32_t c = 0; c + 1 < np; ++c) fchain[static_cast<size_t>(m)].push_back(next++);
    acoef[static_cast<size_t>(m)] = next++;
  }
  std::vector<int32_t> mfactor(static_cast<size_t>(N), -1);  // slot of the common factor F_m
  P.n_slots = next;

  // ---- convolution jobs, each in the earliest layer its operands allow ----
  Builder B;
  std::vector<int32_t> ready(static_cast<size_t>(next), 0);  // layer after which a slot holds its series
  int32_t max_layer = 0;
  auto job = [&](int32_t in1, int32_t in2, int32_t out) {
    const int32_t layer = 1 + std::max(ready[static_cast<size_t>(in1)], ready[static_cast<size_t>(in2)]);
    B.add(in1, in2, out, layer);
    ready[static_cast<size_t>(out)] = layer;
    max_layer = std::max(max_layer, layer);
  };
  for (int32_t v = 0; v < n; ++v)
    for (int32_t q = 2; q <= qmax[static_cast<size_t>(v)]; ++q) job(POW(v, q - 1), Z(v), POW(v, q));
  for (int32_t m = 0; m < N; ++m) {
    if (acoef[static_cast<size_t>(m)] == A(m + 1)) continue;
    std::vector<int32_t> factors;
    for (int32_t t = s.ptr[static_cast<size_t>(m)]; t < s.ptr[static_cast<size_t>(m) + 1]; ++t)
      if (s.exponent(t) >= 2) factors.push_back(POW(s.idx[static_cast<size_t>(t)], s.exponent(t) - 1));
    int32_t f = factors[0];
    for (size_t c = 1; c < factors.size(); ++c) {
      const int32_t o = fchain[static_cast<size_t>(m)][c - 1];
      job(f, factors[c], o);
      f = o;
    }
    mfactor[static_cast<size_t>(m)] = f;
    job(A(m + 1), f, acoef[static_cast<size_t>(m)]);
  }
  P.power_jobs = static_cast<int32_t>(B.jobs.size());
  for (int32_t m = 0; m < N; ++m) {
    const MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    const int32_t* v = s.idx.data() + s.ptr[m];
    const int32_t nk = ms.nk, a = acoef[static_cast<size_t>(m)];
    auto f = [&](int32_t l) { return ms.f0 + l - 1; };  // f_{k,l}, l = 1..nk
    auto b = [&](int32_t l) { return ms.b0 + l - 1; };  // b_{k,l}
    auto c = [&](int32_t l) { return ms.c0 + l - 1; };  // c_{k,l}
    job(a, Z(v[0]), f(1));
    for (int32_t l = 2; l <= nk; ++l) job(f(l - 1), Z(v[l - 1]), f(l));
    if (nk == 2) {
      job(Z(v[1]), a, b(1));
    } else if (nk >= 3) {
      job(Z(v[nk - 1]), Z(v[nk - 2]), b(1));
      for (int32_t l = 2; l <= nk - 2; ++l) job(b(l - 1), Z(v[nk - 1 - l]), b(l));
      job(b(nk - 2), a, ms.bA);
      for (int32_t j = 1; j <= nk - 3; ++j) job(f(j), b(nk - 2 - j), c(j));
      job(f(nk - 2), Z(v[nk - 1]), c(nk - 2));
    }
  }
  P.jobs = B.jobs;
  finalize(P.jobs, P.n_slots);
  P.n_layers = max_layer;
  P.layer_ptr.assign(static_cast<size_t>(max_layer) + 1, 0);
  for (const ConvJob& j : P.jobs) P.layer_ptr[static_cast<size_t>(j.layer)]++;
  for (int32_t L = 1; L <= max_layer; ++L)
    P.layer_ptr[static_cast<size_t>(L)] += P.layer_ptr[static_cast<size_t>(L) - 1];

  // ---- addition stage: value and gradient contributions, monomial order ----
  // every monomial's terms (output, slot, integer factor): the factor of a
  // partial is the variable's exponent
  P.mono_terms.assign(static_cast<size_t>(N), {});
  for (int32_t m = 0; m < N; ++m) {
    const MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    const int32_t* v = s.idx.data() + s.ptr[m];
    const int32_t nk = ms.nk, t0 = s.ptr[m];
    auto e = [&](int32_t j) { return s.exponent(t0 + j); };
    auto& tm = P.mono_terms[static_cast<size_t>(m)];
    tm.push_back({0, ms.f0 + nk - 1, 1});
    if (nk == 1) {
      tm.push_back({1 + v[0], acoef[static_cast<size_t>(m)], e(0)});
    } else if (nk == 2) {
      tm.push_back({1 + v[0], ms.b0, e(0)});  // b_1 = z_{i_2} a
      tm.push_back({1 + v[1], ms.f0, e(1)});  // f_1 = a z_{i_1}
    } else {
      tm.push_back({1 + v[0], ms.bA, e(0)});
      for (int32_t j = 1; j <= nk - 2; ++j) tm.push_back({1 + v[j], ms.c0 + j - 1, e(j)});
      tm.push_back({1 + v[nk - 1], ms.f0 + nk - 2, e(nk - 1)});
    }
  }
  std::vector<std::vector<std::pair<int32_t, int32_t>>> contrib(static_cast<size_t>(n) + 1);
  contrib[0].push_back({0, 1});  // a_0
  for (int32_t m = 0; m < N; ++m)
    for (const auto& t : P.mono_terms[static_cast<size_t>(m)])
      contrib[static_cast<size_t>(t[0])].push_back({t[1], t[2]});
  P.add_ptr.assign(static_cast<size_t>(n) + 2, 0);
  for (size_t o = 0; o < contrib.size(); ++o) P.add_ptr[o + 1] = P.add_ptr[o] + static_cast<int32_t>(contrib[o].size());
  P.add_src.reserve(static_cast<size_t>(P.add_ptr.back()));
  P.add_mult.reserve(static_cast<size_t>(P.add_ptr.back()));
  for (const auto& cl : contrib)
    for (const auto& sm : cl) {
      P.add_src.push_back(sm.first);
      P.add_mult.push_back(sm.second);
    }

  if (!with_vjp || paper_layout) return P;

  // ---- VJP extras: M_k (product of the variables), gradient series, correlations ----
  int32_t nx = P.n_slots;
  P.slot_u = nx++;
  P.mslot.assign(static_cast<size_t>(N), -1);
  Builder V;
  V.jobs = P.jobs;  // forward products first
  for (ConvJob& j : V.jobs) j.dep1 = j.dep2 = -1;
  P.slot_M0 = nx;
  // M_m = prod z_v^{e_v}: the product of the variables (b_{k,nk-2} * z_{i_1}),
  // times the common factor F_m when the monomial has powers
  ready.resize(static_cast<size_t>(nx) + 2 * static_cast<size_t>(N), 0);
  auto vjob = [&](int32_t in1, int32_t in2, int32_t out) {
    const int32_t layer = 1 + std::max(ready[static_cast<size_t>(in1)], ready[static_cast<size_t>(in2)]);
    V.add(in1, in2, out, layer);
    ready[static_cast<size_t>(out)] = layer;
  };
  for (int32_t m = 0; m < N; ++m) {
    const MonoSlots& ms = P.mono[static_cast<size_t>(m)];
    const int32_t* v = s.idx.data() + s.ptr[m];
    int32_t mv;  // product of the variables, each once
    if (ms.nk == 1) {
      mv = Z(v[0]);
    } else if (ms.nk == 2) {
      mv = nx++;
      vjob(Z(v[0]), Z(v[1]), mv);
    } else {
      mv = nx++;
      vjob(ms.b0 + ms.nk - 3, Z(v[0]), mv);  // b_{k,nk-2} * z_{i_1}
    }
    if (mfactor[static_cast<size_t>(m)] >= 0) {
      const int32_t o = nx++;
      vjob(mv, mfactor[static_cast<size_t>(m)], o);
      mv = o;
    }
    P.mslot[static_cast<size_t>(m)] = mv;
  }
  P.slot_g0 = nx;
  nx += n;
  P.slot_r0 = nx;
  nx += N + n;
  P.n_slots_vjp = nx;
  finalize(V.jobs, nx);
  P.vjp_fwd_jobs = static_cast<int32_t>(V.jobs.size());
  for (const ConvJob& j : V.jobs)  // the monomial products alone (their list resolves its own deps)
    if (j.out >= P.slot_M0 && j.out < P.slot_g0)
      P.vjp_mjobs.push_back(ConvJob{j.in1, j.in2, j.out, -1, -1, 0, j.kind, j.layer});
  for (int32_t m = 0; m < N; ++m)
    V.jobs.push_back(ConvJob{P.slot_u, P.mslot[static_cast<size_t>(m)], P.slot_r0 + m, -1, -1, 0, JOB_CORR, 1});
  for (int32_t i = 0; i < n; ++i)
    V.jobs.push_back(ConvJob{P.slot_u, P.slot_g0 + i, P.slot_r0 + N + i, -1, -1, 0, JOB_CORR, 1});
  P.vjp_jobs = V.jobs;
  return P;
}

Program1 compile_system(const Supports& s, const std::vector<int32_t>& poly_ptr, int32_t d, bool with_vjp) {
  Program1 P = compile(s, d, false, with_vjp);
  const int32_t np = static_cast<int32_t>(poly_ptr.size()) - 1, n = s.n;
  P.system_P = np;
  // the constants after every slot of compile's layout (its VJP slots included)
  P.const0 = with_vjp ? P.n_slots_vjp : P.n_slots;
  if (with_vjp) P.n_slots_vjp += np;
  else P.n_slots += np;
  std::vector<std::vector<std::pair<int32_t, int32_t>>> contrib(static_cast<size_t>(np) * (1 + n));
  for (int32_t p = 0; p < np; ++p) {
    contrib[static_cast<size_t>(p)].push_back({P.const0 + p, 1});
    for (int32_t m = poly_ptr[static_cast<size_t>(p)]; m < poly_ptr[static_cast<size_t>(p) + 1]; ++m)
      for (const auto& t : P.mono_terms[static_cast<size_t>(m)]) {
        const size_t o = t[0] == 0 ? static_cast<size_t>(p) : static_cast<size_t>(np + p * n + t[0] - 1);
        contrib[o].push_back({t[1], t[2]});
      }
  }
  P.add_ptr.assign(contrib.size() + 1, 0);
  P.add_src.clear();
  P.add_mult.clear();
  for (size_t o = 0; o < contrib.size(); ++o) {
    for (const auto& sm : contrib[o]) {
      P.add_src.push_back(sm.first);
      P.add_mult.push_back(sm.second);
    }
    P.add_ptr[o + 1] = static_cast<int32_t>(P.add_src.size());
  }
  if (!with_vjp) return P;

  // ---- VJP: one upstream series per polynomial; the correlations of u_p with
  // the monomial products of p and with p's Jacobian series ----
  int32_t nx = P.n_slots_vjp;
  P.slot_up0 = nx;
  nx += np;
  P.slot_J0 = nx;
  nx += np * n;
  P.slot_rJ0 = nx;
  nx += np * n;
  P.n_slots_vjp = nx;
  std::vector<ConvJob> V(P.vjp_jobs.begin(), P.vjp_jobs.begin() + P.vjp_fwd_jobs);  // forward and M_m
  for (int32_t p = 0; p < np; ++p)
    for (int32_t m = poly_ptr[static_cast<size_t>(p)]; m < poly_ptr[static_cast<size_t>(p) + 1]; ++m)
      V.push_back(ConvJob{P.slot_up0 + p, P.mslot[static_cast<size_t>(m)], P.slot_r0 + m, -1, -1, 0, JOB_CORR, 1});
  for (int32_t p = 0; p < np; ++p)
    for (int32_t i = 0; i < n; ++i) {
      const size_t o = static_cast<size_t>(np + p * n + i);
      if (P.add_ptr[o + 1] > P.add_ptr[o])
        V.push_back(ConvJob{P.slot_up0 + p, P.slot_J0 + p * n + i, P.slot_rJ0 + p * n + i, -1, -1, 0, JOB_CORR, 1});
    }
  P.vjp_jobs = V;
  P.slot_u = -1;  // the single upstream slot of compile is not used
  return P;
}

Program1 complexify(const Program1& R) {
  Program1 C;
  C.N = R.N;
  C.n = R.n;
  C.d = R.d;
  C.has_powers = R.has_powers;
  C.n_input_slots = 2 * R.n_input_slots;
  auto re = [](int32_t s) { return 2 * s; };
  auto im = [](int32_t s) { return 2 * s + 1; };
  const bool vjp = !R.vjp_jobs.empty();
  // scratch slots after the doubled layout (its VJP slots included)
  int32_t next = 2 * (vjp ? R.n_slots_vjp : R.n_slots);
  const size_t bound = static_cast<size_t>(next) + 4 * (R.jobs.size() + R.vjp_jobs.size() + R.vjp_mjobs.size());
  // Complex form of a list of real jobs, every job in the earliest layer its
  // operands (within the list) allow: a product x * y becomes xr yr, xi yi,
  // xr yi, xi yr in four scratch slots and re = xr yr - xi yi, im = xr yi + xi yr;
  // a correlation of u with s (the VJP) becomes the correlation with conj(s):
  // re = ur . sr + ui . si, im = ui . sr - ur . si.
  auto cx = [&](std::vector<ConvJob>::const_iterator b, std::vector<ConvJob>::const_iterator e, int32_t* layers,
                int32_t* power) {
    std::vector<int32_t> ready(bound, 0);
    Builder B;
    int32_t max_layer = 0;
    auto job = [&](int32_t in1, int32_t in2, int32_t out, int32_t kind) {
      const int32_t layer = 1 + std::max(ready[static_cast<size_t>(in1)], ready[static_cast<size_t>(in2)]);
      B.add(in1, in2, out, layer, kind);
      ready[static_cast<size_t>(out)] = layer;
      max_layer = std::max(max_layer, layer);
    };
    for (auto it = b; it != e; ++it) {  // producers before consumers
      const ConvJob& r = *it;
      const int32_t t = next;
      next += 4;
      if (r.kind == JOB_CORR) {
        job(re(r.in1), re(r.in2), t, JOB_CORR);
        job(im(r.in1), im(r.in2), t + 1, JOB_CORR);
        job(im(r.in1), re(r.in2), t + 2, JOB_CORR);
        job(re(r.in1), im(r.in2), t + 3, JOB_CORR);
        job(t, t + 1, re(r.out), JOB_ADD);
        job(t + 2, t + 3, im(r.out), JOB_SUB);
      } else {
        job(re(r.in1), re(r.in2), t, JOB_CONV);
        job(im(r.in1), im(r.in2), t + 1, JOB_CONV);
        job(re(r.in1), im(r.in2), t + 2, JOB_CONV);
        job(im(r.in1), re(r.in2), t + 3, JOB_CONV);
        job(t, t + 1, re(r.out), JOB_SUB);
        job(t + 2, t + 3, im(r.out), JOB_ADD);
      }
      if (power && it - b < R.power_jobs) *power += 6;
    }
    finalize(B.jobs, static_cast<int32_t>(bound));
    if (layers) *layers = max_layer;
    return B.jobs;
  };
  int32_t max_layer = 0;
  C.jobs = cx(R.jobs.begin(), R.jobs.end(), &max_layer, &C.power_jobs);
  C.n_slots = next;
  C.n_layers = max_layer;
  C.layer_ptr.assign(static_cast<size_t>(max_layer) + 1, 0);
  for (const ConvJob& j : C.jobs) C.layer_ptr[static_cast<size_t>(j.layer)]++;
  for (int32_t L = 1; L <= max_layer; ++L)
    C.layer_ptr[static_cast<size_t>(L)] += C.layer_ptr[static_cast<size_t>(L) - 1];
  const size_t nout = R.add_ptr.size() - 1;
  C.add_ptr.assign(2 * nout + 1, 0);
  for (size_t o = 0; o < nout; ++o) {
    for (int part = 0; part < 2; ++part) {
      for (int32_t t = R.add_ptr[o]; t < R.add_ptr[o + 1]; ++t) {
        const int32_t s = R.add_src[static_cast<size_t>(t)];
        C.add_src.push_back(part == 0 ? re(s) : im(s));
        C.add_mult.push_back(R.add_mult.empty() ? 1 : R.add_mult[static_cast<size_t>(t)]);
      }
      C.add_ptr[2 * o + part + 1] = static_cast<int32_t>(C.add_src.size());
    }
  }
  if (!vjp) return C;
  // VJP: the forward and monomial products, the monomial products alone, and
  // the correlations, each list layered on its own; the VJP slots keep their
  // real-layout numbers s (the parts live in 2s and 2s + 1)
  std::vector<ConvJob> fwdm = cx(R.vjp_jobs.begin(), R.vjp_jobs.begin() + R.vjp_fwd_jobs, nullptr, nullptr);
  std::vector<ConvJob> corr = cx(R.vjp_jobs.begin() + R.vjp_fwd_jobs, R.vjp_jobs.end(), nullptr, nullptr);
  C.vjp_mjobs = cx(R.vjp_mjobs.begin(), R.vjp_mjobs.end(), nullptr, nullptr);
  C.vjp_fwd_jobs = static_cast<int32_t>(fwdm.size());
  C.vjp_jobs = fwdm;
  C.vjp_jobs.insert(C.vjp_jobs.end(), corr.begin(), corr.end());
  C.slot_u = R.slot_u;
  C.slot_M0 = R.slot_M0;
  C.mslot = R.mslot;
  C.slot_g0 = R.slot_g0;
  C.slot_r0 = R.slot_r0;
  C.n_slots_vjp = next;
  return C;
}

std::vector<int64_t> paper_add_levels(const Supports& s) {
  std::vector<int64_t> sizes;
  sizes.push_back(static_cast<int64_t>(s.N) + 1);  // value: a_0 and N forward products
  std::vector<int64_t> deg(static_cast<size_t>(s.n), 0);
  for (int32_t t = 0; t < (s.N > 0 ? s.ptr[static_cast<size_t>(s.N)] : 0); ++t)
    deg[static_cast<size_t>(s.idx[static_cast<size_t>(t)])]++;
  for (int64_t g : deg) sizes.push_back(g);
  std::vector<int64_t> levels;
  for (;;) {
    int64_t adds = 0;
    for (int64_t& m : sizes) {
      adds += m / 2;
      m -= m / 2;
    }
    if (adds == 0) break;
    levels.push_back(adds);
  }
  return levels;
}

}  // namespace pes
