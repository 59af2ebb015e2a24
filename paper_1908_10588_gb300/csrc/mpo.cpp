// Host-side MPO builder (Eq. MPO) for the vibronic Hamiltonian of Sec. 2.2.
//
// The Hamiltonian arrives as its sum of terms (Eqs. Hel_2, Hvib_2,
// Helvib_2). Each term is a product of local operators on at most three
// chain sites (electronic |i><j|, q, q^2, b^+b, identity). The MPO is the
// finite-state automaton of these products: at every bond a term is either
// not started, finished, or open with a known list of operators already
// placed; open terms with identical placed operators share one channel. The
// coefficient rides on the last operator of each term, so transitions into
// the finished channel are sums over terms and every other transition is a
// plain operator. This gives an exact MPO; no compression is applied.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "common.h"

namespace vb {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *get_error() { return g_err.c_str(); }

vb_status Alloc::get(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (user && user->alloc) {
    *p = user->alloc(bytes, (void *)stream, user->ctx);
    if (!*p) return fail(VB_ENOMEM, "user allocator returned NULL for " + std::to_string(bytes) + " bytes");
    return VB_OK;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? VB_ENOMEM : VB_ECUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return VB_OK;
}

void Alloc::put(void *p) {
  if (!p) return;
  if (user && user->free)
    user->free(p, (void *)stream, user->ctx);
  else
    cudaFree(p);
}

namespace {

std::vector<double> local_op(int code, int d, int n_el) {
  std::vector<double> m((size_t)d * d, 0.0);
  if (code == OPC_ID) {
    for (int i = 0; i < d; ++i) m[(size_t)i * d + i] = 1.0;
  } else if (code >= OPC_E) {
    int ij = code - OPC_E, i = ij / n_el, j = ij % n_el;
    m[(size_t)i * d + j] = 1.0;
  } else if (code == OPC_N) {
    for (int i = 0; i < d; ++i) m[(size_t)i * d + i] = (double)i;
  } else {
    // q = (b + b^+)/sqrt(2), b|n> = sqrt(n)|n-1>
    std::vector<double> q((size_t)d * d, 0.0);
    for (int n = 1; n < d; ++n) {
      double v = std::sqrt((double)n) / std::sqrt(2.0);
      q[(size_t)(n - 1) * d + n] = v;
      q[(size_t)n * d + (n - 1)] = v;
    }
    if (code == OPC_Q) return q;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += q[(size_t)a * d + c] * q[(size_t)c * d + b];
        m[(size_t)a * d + b] = s;
      }
  }
  return m;
}

typedef std::vector<int> Key;  // {-1} not started, {-2} finished, else (pos, code) pairs
const Key K_START = {-1};
const Key K_DONE = {-2};

Key key_at(const Term &t, int b) {
  if (t.f.back().pos <= b) return K_DONE;
  if (t.f.front().pos > b) return K_START;
  Key k;
  for (const Factor &x : t.f)
    if (x.pos <= b) {
      k.push_back(x.pos);
      k.push_back(x.code);
    }
  return k;
}

}  // namespace

vb_status model_terms(const vb_model *m, const char *who, std::vector<Term> &terms) {
  terms.clear();
  const int n_el = m->n_el, nm = m->n_modes;
  auto add = [&](double c, std::vector<Factor> f) {
    if (c != 0.0) terms.push_back(Term{c, std::move(f)});
  };
  for (int i = 0; i < n_el; ++i)
    for (int j = 0; j < n_el; ++j) {
      double h = (i == j) ? m->e0[i] : (m->v0 ? m->v0[i * n_el + j] : 0.0);
      add(h, {{ENT_EL, OPC_E + i * n_el + j}});
    }
  double zpe = 0.0;
  for (int I = 0; I < nm; ++I) {
    add(m->omega[I], {{I, OPC_N}});
    zpe += 0.5 * m->omega[I];
  }
  if (m->include_zpe) add(zpe, {{ENT_POS0, OPC_ID}});
  for (int I = 0; I < nm; ++I)
    for (int i = 0; i < n_el; ++i)
      for (int j = 0; j < n_el; ++j)
        add(m->g1[((size_t)I * n_el + i) * n_el + j], {{ENT_EL, OPC_E + i * n_el + j}, {I, OPC_Q}});
  for (int k = 0; k < m->n_g2; ++k) {
    int I = m->g2_idx[4 * k], J = m->g2_idx[4 * k + 1], i = m->g2_idx[4 * k + 2], j = m->g2_idx[4 * k + 3];
    if (I < 0 || J < 0 || I >= nm || J >= nm || I > J || i < 0 || j < 0 || i >= n_el || j >= n_el)
      return fail(VB_EINVAL, std::string(who) + ": g2 index out of range (need 0 <= I <= J < n_modes)");
    if (I == J)
      add(m->g2_val[k], {{ENT_EL, OPC_E + i * n_el + j}, {I, OPC_Q2}});
    else
      add(m->g2_val[k], {{ENT_EL, OPC_E + i * n_el + j}, {I, OPC_Q}, {J, OPC_Q}});
  }
  return VB_OK;
}

}  // namespace vb

using namespace vb;

extern "C" {

const char *vb_last_error(void) { return get_error(); }
int vb_version(void) { return 100; }

vb_status mpo_build(const vb_model *m, vb_mpo **out) {
  if (!m || !out) return fail(VB_EINVAL, "mpo_build: null argument");
  *out = nullptr;
  if (m->n_el < 1 || m->n_el > 30) return fail(VB_EINVAL, "mpo_build: n_el must be in 1..30");
  if (m->n_modes < 0) return fail(VB_EINVAL, "mpo_build: n_modes < 0");
  if (!m->e0 || (m->n_modes > 0 && (!m->omega || !m->levels || !m->g1)))
    return fail(VB_EINVAL, "mpo_build: missing model array");
  if (m->n_g2 > 0 && (!m->g2_idx || !m->g2_val)) return fail(VB_EINVAL, "mpo_build: missing g2");
  const int n_el = m->n_el, nm = m->n_modes, n = nm + 1;
  // chain order
  std::vector<int> order(n), pos_of_mode(nm, -1);
  int el_pos = -1;
  if (m->site_order) {
    std::vector<int> seen(nm + 1, 0);
    for (int p = 0; p < n; ++p) {
      int s = m->site_order[p];
      if (s < -1 || s >= nm) return fail(VB_EINVAL, "mpo_build: site_order entry out of range");
      if (seen[s + 1]++) return fail(VB_EINVAL, "mpo_build: site_order is not a permutation");
      order[p] = s;
    }
  } else {
    order[0] = -1;
    for (int k = 0; k < nm; ++k) order[k + 1] = k;
  }
  std::vector<int> dims(n);
  for (int p = 0; p < n; ++p) {
    if (order[p] < 0) {
      el_pos = p;
      dims[p] = n_el;
    } else {
      int lv = m->levels[order[p]];
      if (lv < 1 || lv > 4096) return fail(VB_EINVAL, "mpo_build: levels must be in 1..4096");
      dims[p] = lv;
      pos_of_mode[order[p]] = p;
    }
  }
  // ---- terms (Eqs. Hel_2, Hvib_2, Helvib_2), placed on the chain
  std::vector<Term> terms;
  VB_TRY(model_terms(m, "mpo_build", terms));
  for (Term &t : terms) {
    for (Factor &x : t.f) x.pos = x.pos == ENT_EL ? el_pos : x.pos == ENT_POS0 ? 0 : pos_of_mode[x.pos];
    std::sort(t.f.begin(), t.f.end(), [](const Factor &a, const Factor &b) { return a.pos < b.pos; });
  }
  // merge factors on the same site (cannot happen for this model, but keep exact)
  for (Term &t : terms)
    for (size_t a = 1; a < t.f.size(); ++a)
      if (t.f[a].pos == t.f[a - 1].pos) return fail(VB_EINVAL, "mpo_build: two factors on one site");
  if (terms.empty()) return fail(VB_EINVAL, "mpo_build: the Hamiltonian has no terms");

  // ---- channels per bond b = -1 .. n-1
  std::vector<std::map<Key, int>> chan(n + 1);
  for (int b = -1; b < n; ++b) {
    std::set<Key> ks;
    if (b == -1)
      ks.insert(K_START);
    else if (b == n - 1)
      ks.insert(K_DONE);
    else
      for (const Term &t : terms) ks.insert(key_at(t, b));
    std::map<Key, int> &c = chan[b + 1];
    int idx = 0;
    if (ks.count(K_START)) c[K_START] = idx++;
    if (ks.count(K_DONE)) c[K_DONE] = idx++;
    for (const Key &k : ks)
      if (k != K_START && k != K_DONE) c[k] = idx++;
  }

  vb_mpo *mpo = new vb_mpo();
  mpo->n = n;
  mpo->n_el = n_el;
  mpo->el_pos = el_pos;
  mpo->dims = dims;
  mpo->pos_of_mode = pos_of_mode;
  mpo->ch_start.assign(n + 1, -1);
  mpo->ch_done.assign(n + 1, -1);
  for (int b = 0; b <= n; ++b) {
    auto it = chan[b].find(K_START);
    if (it != chan[b].end()) mpo->ch_start[b] = it->second;
    it = chan[b].find(K_DONE);
    if (it != chan[b].end()) mpo->ch_done[b] = it->second;
  }
  mpo->e_zpe = 0.0;
  if (m->include_zpe)
    for (int k = 0; k < nm; ++k) mpo->e_zpe += 0.5 * m->omega[k];
  mpo->sites.resize(n);
  for (int p = 0; p < n; ++p) {
    const std::map<Key, int> &cin = chan[p], &cout = chan[p + 1];
    MpoSite &S = mpo->sites[p];
    const int d = dims[p];
    S.wl = (int)cin.size();
    S.wr = (int)cout.size();
    S.d = d;
    std::map<std::pair<int, int>, std::vector<double>> blk;
    std::map<std::pair<int, int>, bool> summed;
    for (const Term &t : terms) {
      Key kin = key_at(t, p - 1), kout = key_at(t, p);
      if (p == 0) kin = K_START;
      if (p == n - 1) kout = K_DONE;
      int code = OPC_ID;
      bool last = false;
      for (size_t a = 0; a < t.f.size(); ++a)
        if (t.f[a].pos == p) {
          code = t.f[a].code;
          last = (a + 1 == t.f.size());
        }
      std::vector<double> op = local_op(code, d, n_el);
      std::pair<int, int> bk(cin.at(kin), cout.at(kout));
      if (kout == K_DONE && kin != K_DONE) {
        (void)last;
        std::vector<double> &acc = blk[bk];
        if (acc.empty()) acc.assign((size_t)d * d, 0.0);
        for (size_t e = 0; e < op.size(); ++e) acc[e] += t.coef * op[e];
        summed[bk] = true;
      } else {
        auto it = blk.find(bk);
        if (it == blk.end())
          blk[bk] = op;
        else if (it->second != op) {
          delete mpo;
          return fail(VB_EINVAL, "mpo_build: inconsistent automaton transition");
        }
      }
    }
    if (p > 0 && cin.count(K_DONE) && cout.count(K_DONE))
      blk[{cin.at(K_DONE), cout.at(K_DONE)}] = local_op(OPC_ID, d, n_el);
    S.dense.assign((size_t)S.wl * d * d * S.wr, 0.0);
    for (auto &kv : blk) {
      int wi = kv.first.first, wo = kv.first.second;
      const std::vector<double> &op = kv.second;
      bool nonzero = false, ident = true;
      for (int a = 0; a < d; ++a)
        for (int b2 = 0; b2 < d; ++b2) {
          double v = op[(size_t)a * d + b2];
          if (v != 0.0) nonzero = true;
          if (v != (a == b2 ? 1.0 : 0.0)) ident = false;
          S.dense[(((size_t)wi * d + a) * d + b2) * S.wr + wo] = v;
        }
      if (!nonzero) continue;
      MpoBlock B;
      B.win = wi;
      B.wout = wo;
      B.ident = ident ? 1 : 0;
      B.op_off = -1;
      if (!ident) {
        B.op_off = (int)S.csr_ptr.size();  // row-pointer base of this operator
        S.ops.insert(S.ops.end(), op.begin(), op.end());
        for (int a = 0; a < d; ++a) {
          S.csr_ptr.push_back((int)S.csr_col.size());
          for (int b2 = 0; b2 < d; ++b2) {
            const double v = op[(size_t)a * d + b2];
            if (v != 0.0) {
              S.csr_col.push_back(b2);
              S.csr_val.push_back(v);
            }
          }
        }
        S.csr_ptr.push_back((int)S.csr_col.size());
        S.nnz_ops++;
      } else {
        S.n_ident++;
      }
      S.blocks.push_back(B);
    }
    mpo->max_w = std::max(mpo->max_w, std::max(S.wl, S.wr));
    mpo->max_d = std::max(mpo->max_d, d);
  }
  *out = mpo;
  return VB_OK;
}

vb_status mpo_destroy(vb_mpo *mpo) {
  if (!mpo) return VB_OK;
  for (void *p : mpo->dev_allocs) cudaFree(p);
  delete mpo;
  return VB_OK;
}

int mpo_n_sites(const vb_mpo *mpo) { return mpo ? mpo->n : -1; }

vb_status mpo_site_dims(const vb_mpo *mpo, int site, int *w_in, int *d, int *w_out) {
  if (!mpo || site < 0 || site >= mpo->n) return fail(VB_EINVAL, "mpo_site_dims: bad site");
  const MpoSite &S = mpo->sites[site];
  if (w_in) *w_in = S.wl;
  if (d) *d = S.d;
  if (w_out) *w_out = S.wr;
  return VB_OK;
}

vb_status mpo_site_tensor(const vb_mpo *mpo, int site, double *host_out) {
  if (!mpo || site < 0 || site >= mpo->n || !host_out) return fail(VB_EINVAL, "mpo_site_tensor: bad argument");
  const MpoSite &S = mpo->sites[site];
  std::memcpy(host_out, S.dense.data(), S.dense.size() * sizeof(double));
  return VB_OK;
}

}  // extern "C"

namespace vb {

vb_status mpo_upload(const vb_mpo *cmpo) {
  vb_mpo *mpo = const_cast<vb_mpo *>(cmpo);
  int dev = -1;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (mpo->uploaded) {
    if (mpo->device != dev) return fail(VB_ESTATE, "MPO was uploaded to another device");
    return VB_OK;
  }
  auto up = [&](const void *src, size_t bytes, void **dst) -> vb_status {
    VB_TRY_CUDA(cudaMalloc(dst, bytes > 0 ? bytes : 16));
    mpo->dev_allocs.push_back(*dst);
    if (bytes) VB_TRY_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return VB_OK;
  };
  for (MpoSite &S : mpo->sites) {
    VB_TRY(up(S.ops.data(), S.ops.size() * sizeof(double), (void **)&S.d_ops));
    std::vector<float> ops32(S.ops.begin(), S.ops.end());
    VB_TRY(up(ops32.data(), ops32.size() * sizeof(float), (void **)&S.d_ops32));
    VB_TRY(up(S.csr_ptr.data(), S.csr_ptr.size() * sizeof(int), (void **)&S.d_csr_ptr));
    VB_TRY(up(S.csr_col.data(), S.csr_col.size() * sizeof(int), (void **)&S.d_csr_col));
    VB_TRY(up(S.csr_val.data(), S.csr_val.size() * sizeof(double), (void **)&S.d_csr_val));
    std::vector<float> val32(S.csr_val.begin(), S.csr_val.end());
    if (&S == &mpo->sites[0] && mpo->e_zpe != 0.0 && mpo->n > 1) {
      // the mixed form's operators without the zero-point constant: site 0's
      // local block (first channel in, DONE channel out) loses e_zpe on its diagonal
      const int done = mpo->ch_done[1];
      for (const MpoBlock &B : S.blocks)
        if (B.win == 0 && B.wout == done && !B.ident)
          for (int r = 0; r < S.d; ++r)
            for (int k = S.csr_ptr[B.op_off + r]; k < S.csr_ptr[B.op_off + r + 1]; ++k)
              if (S.csr_col[k] == r) val32[k] = (float)(S.csr_val[k] - mpo->e_zpe);
    }
    VB_TRY(up(val32.data(), val32.size() * sizeof(float), (void **)&S.d_csr_val32));
    for (int dir = 0; dir < 2; ++dir) {
      int np = dir == 0 ? S.wr : S.wl;
      std::vector<int> ptr(np + 1, 0), ent;
      std::vector<std::vector<int>> rows(np);
      for (const MpoBlock &B : S.blocks) {
        int prod = dir == 0 ? B.wout : B.win;
        int cons = dir == 0 ? B.win : B.wout;
        rows[prod].push_back(cons);
        rows[prod].push_back(B.ident);
        rows[prod].push_back(B.op_off < 0 ? 0 : B.op_off);
      }
      for (int r = 0; r < np; ++r) {
        ptr[r + 1] = ptr[r] + (int)rows[r].size() / 3;
        ent.insert(ent.end(), rows[r].begin(), rows[r].end());
      }
      int **dp = dir == 0 ? &S.d_fwd_ptr : &S.d_bwd_ptr;
      int **de = dir == 0 ? &S.d_fwd_ent : &S.d_bwd_ent;
      VB_TRY(up(ptr.data(), ptr.size() * sizeof(int), (void **)dp));
      VB_TRY(up(ent.data(), ent.size() * sizeof(int), (void **)de));
    }
  }
  mpo->uploaded = true;
  mpo->device = dev;
  return VB_OK;
}

}  // namespace vb
