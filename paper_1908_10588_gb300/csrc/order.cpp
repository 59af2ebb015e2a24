// Ordering of the chain sites (Sec. 3.1, ordering of local sites; Sec. 4).
//
// The paper finds that the order of the electronic and vibrational sites
// along the chain changes the 2TDVP run time by an order of magnitude, through
// the size of the largest two-site tensor m_{i-1} d_i d_{i+1} m_{i+1} and the
// MPO bond dimension, and recommends placing strongly coupled sites next to
// each other, with the small-basis, strongly entangled sites in the middle of
// the chain and the weakly coupled bath modes at one end. This file turns that
// into a cost model of an order and a search over orders:
//
//  * F: H_eff,2 floating-point operations of one application at every pair,
//    with the MPO of that order (the channel counts and operator blocks of
//    the finite-state-automaton builder, counted here without building the
//    tensors) and the MPS bonds at their saturated size min(m_max, full
//    dimension of either side) — the per-step cost once the bonds have grown
//    (the cost the library's profiler counts for every product);
//  * T: the summed two-site tensor sizes at the same bonds (the Krylov vector
//    work and the split scale with it);
//  * D: the coupling distance sum_{a<b} K_ab |pos_a - pos_b|, with K_ab the
//    dimensionless strength |c| / omega-bar of the terms acting on both a and
//    b (omega-bar the geometric mean frequency of the term's modes). D is the
//    summed coupling strength across all bonds, a proxy for the entanglement
//    the bonds must carry;
//  * the objective J = (w_F F/F0 + w_T T/T0 + w_D D/D0) / (w_F + w_T + w_D),
//    relative to the default order (electronic site first, modes by index),
//    so J = 1 for that order.
//
// Search: all orders for chains of up to 8 sites, else simulated annealing
// (swap, segment reversal and single-site moves; geometric cooling; 20000
// moves up to 32 sites, proportionally fewer beyond, at least 2000) started
// from the better of the default order and the paper's rule of thumb.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "common.h"

namespace vb {
namespace {

// one term with its factors on entities: 0..nm-1 modes, nm the electronic
// site, nm + 1 chain position 0 (the zero-point constant)
struct ETerm {
  int nf;
  int ent[3];
  int code[3];
};

struct OrderModel {
  int n_el = 0, nm = 0, n = 0;
  std::vector<int> dim;        // per entity (0..nm)
  std::vector<ETerm> terms;
  std::vector<double> K;       // (nm + 1)^2 coupling strengths between entities
};

struct Eval {
  double F = 0, T = 0, Tmax = 0, D = 0;
  int max_w = 0;
  std::vector<int> w;          // w[b + 1] = channels at bond b, b = -1 .. n-1
  std::vector<int> nop, nid;   // operator / identity blocks per chain position
};

const uint64_t K_START = (1ull << 47) + 1, K_DONE = (1ull << 47) + 2;

inline uint64_t fcode(int pos, int code) { return ((uint64_t)pos << 11 | (uint64_t)code) + 1; }

bool op_is_zero(int code, int d) { return (code == OPC_Q || code == OPC_Q2 || code == OPC_N) && d == 1; }
bool op_is_ident(int code, int n_el) { return code == OPC_ID || (code == OPC_E && n_el == 1); }

vb_status make_model(const vb_model *m, const char *who, OrderModel &om) {
  if (!m) return fail(VB_EINVAL, std::string(who) + ": null model");
  if (m->n_el < 1 || m->n_el > 30) return fail(VB_EINVAL, std::string(who) + ": n_el must be in 1..30");
  if (m->n_modes < 0 || m->n_modes > 4000) return fail(VB_EINVAL, std::string(who) + ": n_modes out of range");
  if (!m->e0 || (m->n_modes > 0 && (!m->omega || !m->levels || !m->g1)))
    return fail(VB_EINVAL, std::string(who) + ": missing model array");
  if (m->n_g2 > 0 && (!m->g2_idx || !m->g2_val)) return fail(VB_EINVAL, std::string(who) + ": missing g2");
  om.n_el = m->n_el;
  om.nm = m->n_modes;
  om.n = om.nm + 1;
  om.dim.assign(om.n, 0);
  for (int I = 0; I < om.nm; ++I) {
    if (m->levels[I] < 1 || m->levels[I] > 4096)
      return fail(VB_EINVAL, std::string(who) + ": levels must be in 1..4096");
    om.dim[I] = m->levels[I];
  }
  om.dim[om.nm] = om.n_el;
  std::vector<Term> terms;
  VB_TRY(model_terms(m, who, terms));
  if (terms.empty()) return fail(VB_EINVAL, std::string(who) + ": the Hamiltonian has no terms");
  const int ne = om.n;
  om.K.assign((size_t)ne * ne, 0.0);
  for (const Term &t : terms) {
    ETerm e{};
    e.nf = (int)t.f.size();
    double lw = 0.0;
    int nmodes = 0;
    for (int a = 0; a < e.nf; ++a) {
      const int p = t.f[a].pos;
      e.ent[a] = p == ENT_EL ? om.nm : p == ENT_POS0 ? om.nm + 1 : p;
      e.code[a] = t.f[a].code;
      if (p >= 0) {
        if (!(m->omega[p] > 0.0)) continue;
        lw += std::log(m->omega[p]);
        ++nmodes;
      }
    }
    om.terms.push_back(e);
    if (e.nf < 2) continue;
    const double wbar = nmodes ? std::exp(lw / nmodes) : 1.0;
    const double k = std::fabs(t.coef) / wbar;
    for (int a = 0; a < e.nf; ++a)
      for (int b = a + 1; b < e.nf; ++b) {
        const int x = e.ent[a], y = e.ent[b];
        if (x == y || x > om.nm || y > om.nm) continue;
        om.K[(size_t)x * ne + y] += k;
        om.K[(size_t)y * ne + x] += k;
      }
  }
  return VB_OK;
}

// pos[e] = chain position of entity e (e = 0..nm), order[p] = entity at p
void evaluate(const OrderModel &om, const std::vector<int> &order, int m_max, Eval &ev,
              std::vector<uint64_t> &keys, std::vector<std::pair<uint64_t, uint64_t>> &blk) {
  const int n = om.n, ne = om.n;
  std::vector<int> pos(ne), dims(n);
  for (int p = 0; p < n; ++p) {
    pos[order[p]] = p;
    dims[p] = om.dim[order[p]];
  }
  // factors of every term placed and sorted by position
  struct Placed {
    int nf, p[3], code[3];
  };
  std::vector<Placed> pl(om.terms.size());
  int max_first = -1, min_last = n;
  for (size_t t = 0; t < om.terms.size(); ++t) {
    const ETerm &e = om.terms[t];
    Placed &q = pl[t];
    q.nf = e.nf;
    for (int a = 0; a < e.nf; ++a) {
      q.p[a] = e.ent[a] == om.nm + 1 ? 0 : pos[e.ent[a]];
      q.code[a] = e.code[a];
    }
    for (int a = 1; a < q.nf; ++a)  // insertion sort of <= 3 factors
      for (int b = a; b > 0 && q.p[b] < q.p[b - 1]; --b) {
        std::swap(q.p[b], q.p[b - 1]);
        std::swap(q.code[b], q.code[b - 1]);
      }
    max_first = std::max(max_first, q.p[0]);
    min_last = std::min(min_last, q.p[q.nf - 1]);
  }
  // prefix key of a term at bond b (p[0] <= b < p[nf-1])
  auto prefix = [](const Placed &q, int b) {
    uint64_t k = 0;
    for (int a = 0; a < q.nf && q.p[a] <= b; ++a) k = k << 23 | fcode(q.p[a], q.code[a]);
    return k;
  };
  auto key_at = [&](const Placed &q, int b) -> uint64_t {
    if (q.p[q.nf - 1] <= b) return K_DONE;
    if (q.p[0] > b) return K_START;
    return prefix(q, b);
  };
  // ---- channels per bond
  keys.clear();
  for (const Placed &q : pl)
    for (int b = q.p[0]; b < q.p[q.nf - 1]; ++b) keys.push_back((uint64_t)b << 48 | prefix(q, b));
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  ev.w.assign(n + 1, 0);
  ev.w[0] = 1;
  ev.w[n] = 1;
  for (int b = 0; b + 1 < n; ++b) ev.w[b + 1] = (max_first > b) + (min_last <= b);
  for (uint64_t k : keys) ev.w[(k >> 48) + 1]++;
  ev.max_w = *std::max_element(ev.w.begin(), ev.w.end());
  // ---- operator blocks per site: (kin, kout) pairs of the terms acting
  // here, plus the START->START and DONE->DONE pass-through identities
  ev.nop.assign(n, 0);
  ev.nid.assign(n, 0);
  std::vector<std::vector<int>> active(n);
  for (size_t t = 0; t < pl.size(); ++t)
    for (int p = pl[t].p[0]; p <= pl[t].p[pl[t].nf - 1]; ++p) active[p].push_back((int)t);
  for (int p = 0; p < n; ++p) {
    blk.clear();
    const int d = dims[p];
    for (int t : active[p]) {
      const Placed &q = pl[t];
      const uint64_t kin = p == 0 ? K_START : key_at(q, p - 1);
      const uint64_t kout = p == n - 1 ? K_DONE : key_at(q, p);
      int code = -1;
      for (int a = 0; a < q.nf; ++a)
        if (q.p[a] == p) code = q.code[a];
      // low bits of the second word: 1 = identity, 2 = nonzero
      uint64_t flags;
      if (code < 0)
        flags = 3;  // pass-through identity
      else if (kout == K_DONE)
        flags = op_is_zero(code, d) ? 0 : 2;  // summed into the finished channel
      else
        flags = (op_is_zero(code, d) ? 0 : 2) | (op_is_ident(code, om.n_el) ? 1 : 0);
      blk.push_back({kin, kout << 2 | flags});
    }
    if (p + 1 < n && max_first > p) blk.push_back({K_START, K_START << 2 | 3});
    if (p > 0 && min_last <= p - 1) blk.push_back({K_DONE, K_DONE << 2 | 3});
    std::sort(blk.begin(), blk.end());
    for (size_t a = 0; a < blk.size();) {
      size_t b = a;
      bool nonzero = false, ident = true;
      const uint64_t kin = blk[a].first, kout = blk[a].second >> 2;
      const bool summed = kout == K_DONE && kin != K_DONE;
      for (; b < blk.size() && blk[b].first == kin && (blk[b].second >> 2) == kout; ++b) {
        nonzero |= (blk[b].second & 2) != 0;
        ident &= (blk[b].second & 1) != 0;
      }
      if (nonzero) {
        if (ident && !summed)
          ev.nid[p]++;
        else
          ev.nop[p]++;
      }
      a = b;
    }
  }
  // ---- saturated MPS bonds and the cost terms
  std::vector<double> mb(n + 1, 1.0);
  {
    std::vector<double> l(n + 1, 1.0), r(n + 1, 1.0);
    for (int p = 0; p < n; ++p) l[p + 1] = std::min(1e18, l[p] * dims[p]);
    for (int p = n - 1; p >= 0; --p) r[p] = std::min(1e18, r[p + 1] * dims[p]);
    for (int b = 1; b < n; ++b) mb[b] = std::min<double>(m_max, std::min(l[b], r[b]));
  }
  ev.F = ev.T = ev.Tmax = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double mL = mb[i], mR = mb[i + 2];
    const double th = mL * dims[i] * dims[i + 1] * mR;
    ev.F += heff2_flops_of(mL, mR, dims[i], dims[i + 1], ev.w[i], ev.w[i + 2], ev.nop[i], ev.nid[i], ev.nop[i + 1],
                           ev.nid[i + 1]);
    ev.T += th;
    ev.Tmax = std::max(ev.Tmax, th);
  }
  double D = 0.0;
  for (int a = 0; a < ne; ++a)
    for (int b = a + 1; b < ne; ++b) {
      const double k = om.K[(size_t)a * ne + b];
      if (k != 0.0) D += k * std::abs(pos[a] - pos[b]);
    }
  ev.D = D;
}

struct Objective {
  double wF, wT, wD, F0, T0, D0;
  double operator()(const Eval &e) const {
    double s = 0.0, wsum = 0.0;
    if (wF > 0 && F0 > 0) s += wF * e.F / F0, wsum += wF;
    if (wT > 0 && T0 > 0) s += wT * e.T / T0, wsum += wT;
    if (wD > 0 && D0 > 0) s += wD * e.D / D0, wsum += wD;
    return wsum > 0 ? s / wsum : 1.0;
  }
};

vb_status read_opts(const vb_order_opts *o, const char *who, int &m_max, double &wF, double &wT, double &wD) {
  m_max = o ? o->m_max : 64;
  wF = o ? o->w_flops : 1.0;
  wT = o ? o->w_size : 1.0;
  wD = o ? o->w_coupling : 1.0;
  if (m_max < 1) return fail(VB_EINVAL, std::string(who) + ": m_max < 1");
  if (!(wF >= 0) || !(wT >= 0) || !(wD >= 0) || !(wF + wT + wD > 0))
    return fail(VB_EINVAL, std::string(who) + ": weights must be >= 0 and not all zero");
  return VB_OK;
}

// entity order from the C order (-1 = electronic site)
vb_status read_order(const OrderModel &om, const int *order, const char *who, std::vector<int> &out) {
  out.assign(om.n, 0);
  std::vector<int> seen(om.n, 0);
  for (int p = 0; p < om.n; ++p) {
    const int s = order[p];
    if (s < -1 || s >= om.nm) return fail(VB_EINVAL, std::string(who) + ": order entry out of range");
    const int e = s < 0 ? om.nm : s;
    if (seen[e]++) return fail(VB_EINVAL, std::string(who) + ": order is not a permutation");
    out[p] = e;
  }
  return VB_OK;
}

std::vector<int> default_order(const OrderModel &om) {
  std::vector<int> o(om.n);
  o[0] = om.nm;
  for (int k = 0; k < om.nm; ++k) o[k + 1] = k;
  return o;
}

// the paper's rule of thumb: the n_strong modes most strongly coupled to
// the rest, in decreasing strength, alternately right and left of the
// electronic site; the other (bath) modes after them by increasing frequency
std::vector<int> rule_order(const OrderModel &om, const vb_model *m, int n_strong) {
  const int nm = om.nm, ne = om.n;
  std::vector<double> s(nm, 0.0);
  for (int I = 0; I < nm; ++I)
    for (int f = 0; f < ne; ++f) s[I] += om.K[(size_t)I * ne + f];
  std::vector<int> idx(nm);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s[a] > s[b]; });
  n_strong = std::min(std::max(n_strong, 0), nm);
  std::vector<int> left, right;
  for (int r = 0; r < n_strong; ++r) (r % 2 == 0 ? right : left).push_back(idx[r]);
  std::vector<int> bath(idx.begin() + n_strong, idx.end());
  std::stable_sort(bath.begin(), bath.end(), [&](int a, int b) { return m->omega[a] < m->omega[b]; });
  std::vector<int> o(left.rbegin(), left.rend());
  o.push_back(nm);
  o.insert(o.end(), right.begin(), right.end());
  o.insert(o.end(), bath.begin(), bath.end());
  return o;
}

inline uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

void fill_cost(const Eval &e, double J, vb_order_cost *out) {
  if (!out) return;
  out->heff_flops = e.F;
  out->tensor_elems = e.T;
  out->max_tensor = e.Tmax;
  out->coupling_dist = e.D;
  out->objective = J;
  out->max_w = e.max_w;
}

}  // namespace
}  // namespace vb

using namespace vb;

extern "C" {

vb_status vb_site_order_cost(const vb_model *model, const int *order, const vb_order_opts *opts,
                             vb_order_cost *out, int *mpo_bonds, int *site_blocks) {
  const char *who = "vb_site_order_cost";
  OrderModel om;
  VB_TRY(make_model(model, who, om));
  int m_max;
  double wF, wT, wD;
  VB_TRY(read_opts(opts, who, m_max, wF, wT, wD));
  std::vector<int> ord;
  if (order || model->site_order)
    VB_TRY(read_order(om, order ? order : model->site_order, who, ord));
  else
    ord = default_order(om);
  std::vector<uint64_t> keys;
  std::vector<std::pair<uint64_t, uint64_t>> blk;
  Eval e, e0;
  evaluate(om, ord, m_max, e, keys, blk);
  evaluate(om, default_order(om), m_max, e0, keys, blk);
  Objective J{wF, wT, wD, e0.F, e0.T, e0.D};
  fill_cost(e, J(e), out);
  if (mpo_bonds)
    for (int b = 0; b + 1 < om.n; ++b) mpo_bonds[b] = e.w[b + 1];
  if (site_blocks)
    for (int p = 0; p < om.n; ++p) {
      site_blocks[2 * p] = e.nop[p];
      site_blocks[2 * p + 1] = e.nid[p];
    }
  return VB_OK;
}

vb_status vb_site_order_rule(const vb_model *model, int n_strong, int *order_out) {
  const char *who = "vb_site_order_rule";
  if (!order_out) return fail(VB_EINVAL, std::string(who) + ": null order_out");
  OrderModel om;
  VB_TRY(make_model(model, who, om));
  std::vector<int> o = rule_order(om, model, n_strong);
  for (int p = 0; p < om.n; ++p) order_out[p] = o[p] == om.nm ? -1 : o[p];
  return VB_OK;
}

vb_status vb_site_order_search(const vb_model *model, const vb_order_opts *opts, int *order_out,
                               vb_order_cost *out) {
  const char *who = "vb_site_order_search";
  if (!order_out) return fail(VB_EINVAL, std::string(who) + ": null order_out");
  OrderModel om;
  VB_TRY(make_model(model, who, om));
  int m_max;
  double wF, wT, wD;
  VB_TRY(read_opts(opts, who, m_max, wF, wT, wD));
  const int n = om.n;
  int iters = opts ? opts->iters : 0;
  const int n_strong = opts && opts->n_strong > 0 ? opts->n_strong : 4;
  uint64_t rng = opts ? opts->seed : 0;
  if (iters < 0 && n > 10) return fail(VB_EINVAL, std::string(who) + ": exhaustive search needs <= 10 sites");
  // default: every order up to 8 sites; else 20000 moves, fewer on long
  // chains (one evaluation costs O(terms x chain length))
  if (iters == 0) iters = n <= 8 ? -1 : std::max(2000, (int)(20000LL * std::min(n, 32) / n));

  std::vector<uint64_t> keys;
  std::vector<std::pair<uint64_t, uint64_t>> blk;
  Eval e, e0;
  std::vector<int> d0 = default_order(om);
  evaluate(om, d0, m_max, e0, keys, blk);
  Objective J{wF, wT, wD, e0.F, e0.T, e0.D};
  std::vector<int> best = d0;
  double jbest = J(e0);
  Eval ebest = e0;

  if (iters < 0) {
    // every order, in lexicographic order of entity ids
    std::vector<int> o(n);
    std::iota(o.begin(), o.end(), 0);
    do {
      evaluate(om, o, m_max, e, keys, blk);
      const double j = J(e);
      if (j < jbest) jbest = j, best = o, ebest = e;
    } while (std::next_permutation(o.begin(), o.end()));
  } else if (n > 1) {
    std::vector<int> cur = rule_order(om, model, n_strong);
    evaluate(om, cur, m_max, e, keys, blk);
    double jcur = J(e);
    if (jcur < jbest) jbest = jcur, best = cur, ebest = e;
    else cur = best, jcur = jbest;
    const double t0 = 0.02, t1 = 1e-5;
    std::vector<int> cand;
    for (int it = 0; it < iters; ++it) {
      const double temp = t0 * std::pow(t1 / t0, (double)it / std::max(1, iters - 1));
      cand = cur;
      const int a = (int)(splitmix(rng) % n);
      int b = (int)(splitmix(rng) % (n - 1));
      if (b >= a) ++b;
      const int lo = std::min(a, b), hi = std::max(a, b);
      switch (splitmix(rng) % 3) {
        case 0: std::swap(cand[a], cand[b]); break;
        case 1: std::reverse(cand.begin() + lo, cand.begin() + hi + 1); break;
        default: {
          const int x = cand[a];
          cand.erase(cand.begin() + a);
          cand.insert(cand.begin() + b, x);
        }
      }
      evaluate(om, cand, m_max, e, keys, blk);
      const double j = J(e);
      const double u = (double)(splitmix(rng) >> 11) * (1.0 / 9007199254740992.0);
      if (j <= jcur || u < std::exp((jcur - j) / temp)) {
        cur.swap(cand);
        jcur = j;
        if (j < jbest) jbest = j, best = cur, ebest = e;
      }
    }
  }
  for (int p = 0; p < n; ++p) order_out[p] = best[p] == om.nm ? -1 : best[p];
  fill_cost(ebest, jbest, out);
  return VB_OK;
}

}  // extern "C"
