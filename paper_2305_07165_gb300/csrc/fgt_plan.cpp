// Host planner and C ABI of the box FGT (Algorithm 4, Section 4.2; periodic
// variant Section 5).  Builds, once per (tree, delta, tol, bc):
//   - the validated box tree (leaves tile B, 2:1 balance with corners,
//     Definition treedefs; across the wrap for periodic problems),
//   - the cutoff level l_c and the plane-wave parameters of Theorem 1
//     (eqs. (D0), (pwterms)) or the Fourier parameters of Section 2.2,
//   - the flags f(B) (Definition fflagdef), the P-list (out->in gather at
//     l_c) and the D-list (near-field pairs) work lists,
//   - the FP64 1D tables of Section 4.1 (T_val->pw, T_pw->pot with the
//     separable shift phases folded in, T_val->pot for the 11 neighbour
//     offsets, the diagonal shift phase vectors),
// uploads them and sizes the expansion workspace.  Execution is enqueued by
// fgt_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/fgt.h"
#include "fgt_exec.h"
#include "fgt_internal.h"
#include "fgt_tables.h"

using cd = std::complex<double>;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
thread_local std::string g_err;

fgt_status fail(fgt_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

fgt_status cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return FGT_ERR_CUDA;
}

inline uint64_t box_key(int level, const int32_t *c) {
  return ((uint64_t)level << 57) | (uint64_t)c[0] | ((uint64_t)c[1] << 19) | ((uint64_t)c[2] << 38);
}

struct Box {
  int32_t level = 0;
  int32_t c[3] = {0, 0, 0};
  int32_t parent = -1;
  int32_t child0 = -1;   // first of 2^d consecutive entries in Plan::children, -1 for a leaf
  int64_t leaf = -1;     // leaf index, -1 for an internal box
  int32_t f = 0;         // Definition fflagdef
  int32_t slot = -1;     // expansion slot
  int32_t mind = 0, maxd = 0;  // min / max depth of the leaves below, relative to this box
};

// Bump allocator over one device allocation.
struct DevPack {
  std::vector<std::pair<size_t, std::vector<unsigned char>>> parts;
  std::vector<std::string> names;
  size_t size = 0;
  size_t add(const std::string &name, const void *p, size_t bytes) {
    size_t off = (size + 255) & ~(size_t)255;
    std::vector<unsigned char> v(bytes);
    if (bytes) std::memcpy(v.data(), p, bytes);
    parts.emplace_back(off, std::move(v));
    names.push_back(name);
    size = off + bytes;
    return off;
  }
  template <typename T>
  size_t add(const std::string &name, const std::vector<T> &v) {
    return add(name, v.data(), v.size() * sizeof(T));
  }
};

}  // namespace

struct fgt_plan {
  int d = 0, k = 0, bc = 0, prec = FGT_PREC_FP64, mode = FGT_MODE_FUSED;
  bool f32() const { return prec == FGT_PREC_SPLIT; }  // FP32 expansions and contractions
  // launch-shape knobs (fgt_plan_autotune picks them by timing; these defaults measured best
  // on the 3D adaptive benchmark workload)
  fgt_tuning tune{8, 8, 4, 2, 0.0};  // form_group, eval_rows16, eval_rows_large, near_phase, ms
  double delta = 0, tol = 0, eps_pw = 0;
  // parameters
  int lc = 0, fourier = 0, n_f = 0, n_p = 0, M = 0, n1 = 0, nh = 0, lmax = 0;
  double D0 = 0, R = 0, h = 0, kappa = 0;
  std::vector<double> wmode;  // weight of mode index a in [0, n1), m = a - (M - 1)
  // tree
  int64_t n_leaves = 0;
  std::vector<int32_t> leaf_level, leaf_coord;
  // optional output tree (refines the source tree): u is evaluated at its leaves' nodes
  int64_t n_out = 0;                           // 0: the source tree's own leaves
  std::vector<int32_t> out_level, out_coord;
  std::vector<int64_t> out_src;                // source leaf containing each output leaf
  int64_t n_targets() const { return n_out > 0 ? n_out : n_leaves; }
  std::vector<Box> boxes;
  std::vector<int32_t> children;
  std::unordered_map<uint64_t, int32_t> index;
  std::vector<int32_t> leaf_box;
  std::vector<std::vector<int32_t>> by_level;
  // quadrature
  std::vector<double> eta, weta, Tvp;
  // device state
  bool dirty = true;
  void *dev = nullptr;
  size_t dev_bytes = 0;
  void *work = nullptr;
  size_t work_bytes = 0;
  double *stage = nullptr;  // host-path staging: sigma [n_leaves k^d], then u [n_targets k^d]
  // pipelined host path: copy-in and copy-out streams, two staging slots (sigma then u each), per
  // slot the events "input arrived", "transform done" and "output copied out"
  cudaStream_t hp_in = nullptr, hp_out = nullptr;
  cudaEvent_t hp_in_ev[2] = {}, hp_done_ev[2] = {}, hp_free_ev[2] = {};
  double *hp_stage = nullptr;
  size_t hp_elems = 0;     // per slot
  int hp_next = 0;         // slot of the next call
  bool hp_used[2] = {false, false};
  size_t stage_elems = 0;
  bool host_only = false;   // planned without a device (inspection only)
  bool tc_eval = false;     // split precision: evaluate with the tensor-core kernel (FGT_TC_EVAL=1)
  bool tc_eval4 = false;    // split precision: stages 2-3 of the evaluation on the tensor cores
  bool eval5 = false;       // 3D: evaluation with the half-range axis contracted last
  bool tc_eval6 = false;    // split precision, 3D, K <= 16: evaluation stage 1 on tcgen05 (FGT_TC_EVAL6=1)
  bool eval7 = false;       // split precision, 3D: every evaluation stage on tcgen05 (eval7_kernel)
  bool form7 = false;       // split precision, 3D: every form stage on tcgen05 (form7_kernel), K = 16, 32
  bool form7_k8 = false;    // and for K = 8 blocks
  bool ozaki = true;        // FP64_TC, 3D: form and evaluation as sliced FP64 stages on the BF16 tensor cores
  bool gather2_fp64 = true;   // FP64 expansions: the run-form gather too (FGT_GATHER2=0: the per-anchor one)
  bool gather3 = true;        // 3D, every cutoff-level box an anchor: the stencil-form gather (FGT_GATHER3=0: off)
  cudaStream_t side[fgt::kSides] = {};     // near field and concurrent per-size launches
  cudaEvent_t fork_ev[fgt::kSides] = {}, join_ev[fgt::kSides] = {};
  DevPack host_pack;        // host copy of the uploaded lists and tables (kept for host-only plans)
  fgt::ExecDesc ex;
  fgt_plan_info info{};
  // per-phase profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  // host copies kept for flop accounting
  int64_t n_near_pairs = 0, n_gather_pairs = 0, n_blocks = 0;

  int32_t find(int level, const int32_t *c) const {
    auto it = index.find(box_key(level, c));
    return it == index.end() ? -1 : it->second;
  }
  int np() const { return d == 3 ? k * k * k : k * k; }
  ~fgt_plan() {
    if (hp_out) cudaStreamSynchronize(hp_out);  // pipelined host calls still copying out
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < fgt::kSides; ++i) {
      if (fork_ev[i]) cudaEventDestroy(fork_ev[i]);
      if (join_ev[i]) cudaEventDestroy(join_ev[i]);
      if (side[i]) cudaStreamDestroy(side[i]);
    }
    if (dev) cudaFree(dev);
    if (work) cudaFree(work);
    if (stage) cudaFree(stage);
    for (int i = 0; i < 2; ++i) {
      if (hp_in_ev[i]) cudaEventDestroy(hp_in_ev[i]);
      if (hp_done_ev[i]) cudaEventDestroy(hp_done_ev[i]);
      if (hp_free_ev[i]) cudaEventDestroy(hp_free_ev[i]);
    }
    if (hp_in) cudaStreamDestroy(hp_in);
    if (hp_out) cudaStreamDestroy(hp_out);
    if (hp_stage) cudaFree(hp_stage);
  }
};

namespace {

// ---------------------------------------------------------------------------- parameters

void choose_params(double delta, double eps, int bc, int &lc, double &D0, double &R, double &h, int &M,
                   int &n_p, int &fourier) {
  D0 = std::sqrt(std::log(3.0 / eps));
  const double cut = D0 * std::sqrt(delta);
  // l_c: the finest level whose boxes are still at least D0 sqrt(delta) wide, so that only
  // neighbouring boxes interact above the tolerance (Section 3, cutoff level)
  lc = 0;
  while (lc < fgt::kMaxLevel && std::ldexp(1.0, -(lc + 1)) >= cut) ++lc;
  // range covered by the plane waves: |x_i - y_i| <= 2 L_c between colleagues (just L_0 = 1
  // for the lone root when l_c = 0); Theorem 1 needs R >= D0
  const double span = (lc == 0) ? 1.0 : 2.0 * std::ldexp(1.0, -lc);
  R = std::max(span / std::sqrt(delta), D0);
  h = 2.0 * kPi / (R + D0);
  M = (int)std::ceil(D0 * (R + D0) / kPi);
  n_p = (int)std::ceil(std::sqrt(std::log(1.0 / eps)) / (kPi * std::sqrt(delta)));
  fourier = (bc == FGT_BC_PERIODIC && lc <= 1) ? 1 : 0;
}

// ---------------------------------------------------------------------------- tree

fgt_status build_tree(fgt_plan &P) {
  const int d = P.d;
  const int64_t n = P.n_leaves;
  P.boxes.reserve((size_t)(n * 1.2) + 16);
  P.leaf_box.assign(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    const int lev = P.leaf_level[i];
    if (lev < 0 || lev > fgt::kMaxLevel)
      return fail(FGT_ERR_TREE, "leaf " + std::to_string(i) + ": level out of range");
    Box b;
    b.level = lev;
    for (int a = 0; a < d; ++a) {
      const int32_t c = P.leaf_coord[i * d + a];
      if (c < 0 || c >= (1 << lev)) return fail(FGT_ERR_TREE, "leaf " + std::to_string(i) + ": coordinate out of range");
      b.c[a] = c;
    }
    b.leaf = i;
    const uint64_t key = box_key(lev, b.c);
    if (P.index.count(key)) return fail(FGT_ERR_TREE, "leaf " + std::to_string(i) + " duplicates another leaf");
    P.index[key] = (int32_t)P.boxes.size();
    P.leaf_box[i] = (int32_t)P.boxes.size();
    P.boxes.push_back(b);
  }
  // ancestors
  for (int64_t i = 0; i < n; ++i) {
    Box cur = P.boxes[P.leaf_box[i]];
    while (cur.level > 0) {
      Box par;
      par.level = cur.level - 1;
      for (int a = 0; a < d; ++a) par.c[a] = cur.c[a] >> 1;
      const uint64_t key = box_key(par.level, par.c);
      auto it = P.index.find(key);
      if (it != P.index.end()) {
        if (P.boxes[it->second].leaf >= 0)
          return fail(FGT_ERR_TREE, "leaf " + std::to_string(i) + " overlaps leaf " +
                                        std::to_string(P.boxes[it->second].leaf));
        break;
      }
      P.index[key] = (int32_t)P.boxes.size();
      P.boxes.push_back(par);
      cur = par;
    }
  }
  // parent / child links
  const int nc = 1 << d;
  std::vector<int> nkids(P.boxes.size(), 0);
  for (size_t b = 0; b < P.boxes.size(); ++b) {
    Box &bx = P.boxes[b];
    if (bx.level == 0) continue;
    int32_t pc[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) pc[a] = bx.c[a] >> 1;
    bx.parent = P.find(bx.level - 1, pc);
    nkids[bx.parent]++;
  }
  const int32_t root_c[3] = {0, 0, 0};
  if (P.find(0, root_c) < 0) return fail(FGT_ERR_TREE, "empty tree");
  for (size_t b = 0; b < P.boxes.size(); ++b) {
    if (P.boxes[b].leaf >= 0) continue;
    if (nkids[b] != nc) return fail(FGT_ERR_TREE, "leaves do not tile B (a box has missing children)");
    P.boxes[b].child0 = (int32_t)P.children.size();
    for (int c = 0; c < nc; ++c) {
      int32_t cc[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) cc[a] = 2 * P.boxes[b].c[a] + ((c >> a) & 1);
      P.children.push_back(P.find(P.boxes[b].level + 1, cc));
    }
  }
  // levels, depth ranges
  P.lmax = 0;
  for (const Box &b : P.boxes) P.lmax = std::max(P.lmax, b.level);
  P.by_level.assign(P.lmax + 1, {});
  for (size_t b = 0; b < P.boxes.size(); ++b) P.by_level[P.boxes[b].level].push_back((int32_t)b);
  for (int l = P.lmax; l >= 0; --l)
    for (int32_t b : P.by_level[l]) {
      Box &bx = P.boxes[b];
      if (bx.leaf >= 0) { bx.mind = bx.maxd = 0; continue; }
      int mn = 1 << 30, mx = 0;
      for (int c = 0; c < nc; ++c) {
        const Box &ch = P.boxes[P.children[bx.child0 + c]];
        mn = std::min(mn, ch.mind + 1);
        mx = std::max(mx, ch.maxd + 1);
      }
      bx.mind = mn;
      bx.maxd = mx;
    }
  // 2:1 balance across shared boundary points, corners included
  const bool per = P.bc == FGT_BC_PERIODIC;
  int noff = 1;
  for (int a = 0; a < d; ++a) noff *= 3;
  for (int64_t i = 0; i < n; ++i) {
    const Box &T = P.boxes[P.leaf_box[i]];
    const int l = T.level, nb = 1 << l;
    for (int oc = 0; oc < noff; ++oc) {
      int o[3] = {0, 0, 0}, q[3] = {0, 0, 0};
      bool ok = true, zero = true;
      for (int a = 0, r = oc; a < d; ++a, r /= 3) {
        o[a] = r % 3 - 1;
        if (o[a]) zero = false;
        int v = T.c[a] + o[a];
        if (v < 0 || v >= nb) {
          if (!per) { ok = false; break; }
          v = (v + nb) % nb;
        }
        q[a] = v;
      }
      if (!ok || zero) continue;
      const int32_t nbx = P.find(l, q);
      if (nbx >= 0) {
        const Box &N = P.boxes[nbx];
        if (N.leaf >= 0) continue;
        for (int c = 0; c < nc; ++c) {
          bool touch = true;
          for (int a = 0; a < d; ++a) {
            const int bit = (c >> a) & 1;
            if ((o[a] == 1 && bit != 0) || (o[a] == -1 && bit != 1)) touch = false;
          }
          if (touch && P.boxes[P.children[N.child0 + c]].leaf < 0)
            return fail(FGT_ERR_TREE, "tree is not 2:1 balanced (leaf " + std::to_string(i) +
                                          " touches leaves two or more levels finer)");
        }
      } else {
        int32_t pq[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) pq[a] = q[a] >> 1;
        const int32_t pb = (l >= 1) ? P.find(l - 1, pq) : -1;
        if (pb < 0 || P.boxes[pb].leaf < 0)
          return fail(FGT_ERR_TREE, "tree is not 2:1 balanced (leaf " + std::to_string(i) +
                                        " touches a leaf two or more levels coarser)");
      }
    }
  }
  return FGT_OK;
}

// ---------------------------------------------------------------------------- tables

// Form matrix of a leaf at level l whose expansion centre is offset by `shift` from the leaf
// centre: F[a][j] = w_a (L/2) exp(-i kappa m_a shift) sum_n I[P_n](-kappa m_a L/2) Tvp[n][j]
// (Lemma pwbox with the separable T_c->p shift folded in).
void form_matrix(const fgt_plan &P, int l, double shift, cd *F) {
  const int k = P.k;
  const double L = std::ldexp(1.0, -l);
  double re[72], im[72];
  for (int a = 0; a < P.n1; ++a) {
    const int m = a - (P.M - 1);
    const double t = -P.kappa * m * 0.5 * L;
    fgt::legendre_fourier_integrals(t, k - 1, re, im);
    const cd ph = std::polar(P.wmode[a] * 0.5 * L, -P.kappa * m * shift);
    for (int j = 0; j < k; ++j) {
      cd s = 0;
      for (int nn = 0; nn < k; ++nn) s += cd(re[nn], im[nn]) * P.Tvp[nn * k + j];
      F[a * k + j] = ph * s;
    }
  }
}

// Evaluation matrix: E[t][a] = exp(i kappa m_a ((L/2) eta_t + shift)) (Lemma thm:pweval, T_pw->pot
// with T_p->c folded in).
void eval_matrix(const fgt_plan &P, int l, double shift, cd *E) {
  const double L = std::ldexp(1.0, -l);
  for (int t = 0; t < P.k; ++t)
    for (int a = 0; a < P.n1; ++a) {
      const int m = a - (P.M - 1);
      E[t * P.n1 + a] = std::polar(1.0, P.kappa * m * (0.5 * L * P.eta[t] + shift));
    }
}

// Near-field table (Lemma directbox): K[t][j] = int_S exp(-(x_t - y)^2/delta) l_j(y) dy for a
// source of level ls and a target whose centre is offset by tau0 source half-sides and whose side
// is ratio times the source side; = (L/2) sum_n J_lambda[P_n](tau_t) Tvp[n][j], lambda =
// 2 sqrt(delta)/L, tau_t = tau0 + ratio eta_t.
void near_table(const fgt_plan &P, int ls, double tau0, double ratio, double *K) {
  const int k = P.k;
  const double L = std::ldexp(1.0, -ls);
  const double lam = 2.0 * std::sqrt(P.delta) / L;
  double J[72];
  for (int t = 0; t < k; ++t) {
    const double tau = tau0 + ratio * P.eta[t];
    fgt::gauss_legendre_integrals(lam, tau, k - 1, J);
    for (int j = 0; j < k; ++j) {
      double s = 0;
      for (int nn = 0; nn < k; ++nn) s += J[nn] * P.Tvp[nn * k + j];
      K[t * k + j] = 0.5 * L * s;
    }
  }
}

// kind of a near-field table from the level difference and the centre offset in quarter source sides
int near_kind(int ldiff, int o4) {
  if (ldiff == 0) return o4 == -4 ? 0 : (o4 == 0 ? 1 : (o4 == 4 ? 2 : -1));
  if (ldiff == 1) return o4 == -3 ? 3 : (o4 == -1 ? 4 : (o4 == 1 ? 5 : (o4 == 3 ? 6 : -1)));
  if (ldiff == -1) return o4 == -6 ? 7 : (o4 == -2 ? 8 : (o4 == 2 ? 9 : (o4 == 6 ? 10 : -1)));
  return -1;
}

void kind_geometry(int kind, int &o4, int &ldiff, double &ratio) {
  static const int o4s[11] = {-4, 0, 4, -3, -1, 1, 3, -6, -2, 2, 6};
  o4 = o4s[kind];
  ldiff = kind < 3 ? 0 : (kind < 7 ? 1 : -1);
  ratio = ldiff == 0 ? 1.0 : (ldiff == 1 ? 0.5 : 2.0);
}

template <typename C>
void push_complex(std::vector<C> &dst, const cd *src, size_t n) {
  for (size_t i = 0; i < n; ++i) dst.push_back(C{(decltype(C::x))src[i].real(), (decltype(C::x))src[i].imag()});
}

// ---------------------------------------------------------------------------- device state

struct MatKey {
  int l, la, obase, dl;
  bool operator<(const MatKey &o) const { return std::tie(l, la, obase, dl) < std::tie(o.l, o.la, o.obase, o.dl); }
};

// Algorithmic flop counts of one execution (real flops; complex MAC = 8, real x complex = 4).
void fill_flops(fgt_plan &P, const fgt::ExecDesc &ex, const std::vector<fgt::Block> &blocks, int64_t shift_flops,
                size_t n_anchor) {
  const int d = P.d, k = P.k;
  const int64_t n1 = P.n1, nh = P.nh;
  fgt_plan_info &I = P.info;
  I.n_anchor_boxes = P.fourier ? 1 : (int64_t)n_anchor;
  I.n_form_blocks = ex.n_blocks;
  I.n_direct_pairs = P.n_near_pairs;
  I.n_gather_pairs = P.n_gather_pairs;
  int64_t ff = 0, ef = 0;
  // evaluation flops in the contraction order of the kernel that takes the block: the half-range
  // axis last (eval5 ranges) or first (all others)
  auto half_range_last = [&](int64_t K) {
    if (ex.oz) return true;  // the sliced stages contract m1, m2, then m3
    for (const fgt::LaunchRange &lr : ex.e2_ranges)
      if (lr.K == K) return lr.tensor == 3 || lr.tensor == 7;
    return false;
  };
  for (const fgt::Block &b : blocks) {
    const int64_t K = b.K;
    if (d == 3) {
      ff += 4 * nh * K * K * K + 8 * nh * n1 * K * K + 8 * nh * n1 * n1 * K;
      ef += half_range_last(K) ? 8 * K * nh * n1 * n1 + 8 * K * K * nh * n1 + 4 * K * K * K * nh
                               : K * (8 * nh * n1 * n1 + 8 * K * n1 * n1 + 4 * K * K * n1);
    } else {
      ff += 4 * nh * K * K + 8 * nh * n1 * K;
      ef += K * (8 * nh * n1 + 4 * K * n1);
    }
  }
  I.form_flops = ff;
  I.eval_flops = ef;
  I.gather_flops = 8 * P.n_gather_pairs * ex.slot_size + shift_flops;
  I.direct_flops = P.n_near_pairs * 2 * d * (int64_t)P.np() * k;
  I.prec = P.prec;
  I.mode = P.mode;
  I.launches = fgt::launches_per_transform(ex);
  I.n_tc_eval_blocks = 0;
  for (const fgt::LaunchRange &lr : ex.e2_ranges)
    if (lr.tensor == 7) I.n_tc_eval_blocks += lr.count;
  I.n_tc_form_blocks = 0;
  for (const fgt::LaunchRange &lr : ex.f2_ranges)
    if (lr.tensor == 7) I.n_tc_form_blocks += lr.count;
  I.n_sliced_jobs = 0;
  if (ex.oz)
    for (int kind = 0; kind < 6; ++kind) I.n_sliced_jobs += ex.oz_njobs[kind];
}

template <typename C>
fgt_status prepare_typed(fgt_plan &P, bool upload) {
  const int d = P.d, k = P.k, n1 = P.n1, nh = P.nh, nc = 1 << d;
  const bool hier = P.mode == FGT_MODE_HIERARCHICAL && !P.fourier;
  DevPack pack;
  fgt::ExecDesc ex;
  ex.d = d; ex.k = k; ex.n1 = n1; ex.nh = nh; ex.prec = P.f32() ? 1 : 0; ex.fourier = P.fourier;
  ex.tc64 = P.prec == FGT_PREC_FP64_TC ? 1 : 0;
  ex.slot_size = (int64_t)nh * (d == 3 ? (int64_t)n1 * n1 : (int64_t)n1);

  // ---- slots and anchors
  for (Box &b : P.boxes) b.slot = -1;
  std::vector<int32_t> anchors;  // boxes owning an expansion at the cutoff level (root in Fourier mode)
  int32_t nslots = 0;
  if (P.fourier) {
    const int32_t rc[3] = {0, 0, 0};
    const int32_t root = P.find(0, rc);
    P.boxes[root].slot = nslots++;
    anchors.push_back(root);
  } else {
    if (P.lc <= P.lmax)
      for (int32_t b : P.by_level[P.lc])
        if (P.boxes[b].f) anchors.push_back(b);
    if (hier) {
      for (int l = P.lc; l <= P.lmax; ++l)
        for (int32_t b : P.by_level[l])
          if (P.boxes[b].f) P.boxes[b].slot = nslots++;
    } else {
      for (int32_t a : anchors) P.boxes[a].slot = nslots++;
    }
  }
  ex.n_phi_slots = nslots;
  ex.n_psi_slots = P.fourier ? 0 : nslots;

  // ---- smem-limited block size
  const int smax = upload ? fgt::max_dynamic_smem() : 232448;  // sm_103 opt-in limit without a device
  int dlcap = 0;
  // K = 2^dl k <= 64 (blocks of K > 16 use the per-plane form and per-row evaluation kernels)
  while (((2 << dlcap) * k) <= 64) ++dlcap;
  auto fits = [&](int dl) {
    const int K = (1 << dl) * k;
    return fgt::form_smem_bytes(d, K, n1, P.f32()) <= (size_t)smax &&
           fgt::eval_smem_bytes(d, K, n1, P.f32()) <= (size_t)smax;
  };
  while (dlcap > 0 && !fits(dlcap)) --dlcap;
  if (!fits(0)) return fail(FGT_ERR_ARG, "expansion too large for shared memory (n_f too big for this k)");
  if (hier) dlcap = 0;

  // ---- blocks
  std::vector<fgt::Block> blocks;
  std::vector<int64_t> bleaves;
  std::map<MatKey, int32_t> matid;
  std::vector<C> Ff, Fh, Ef, Eh;
  int32_t nmat = 0;
  std::vector<cd> Fb((size_t)n1 * k), Eb((size_t)k * n1);
  auto get_mat = [&](int l, int la, int obase, int dl, double anchor_lo) -> int32_t {
    MatKey key{l, la, obase, dl};
    auto it = matid.find(key);
    if (it != matid.end()) return it->second;
    const int32_t id = nmat;
    const double L = std::ldexp(1.0, -l), La = std::ldexp(1.0, -la);
    for (int o = obase; o < obase + (1 << dl); ++o) {
      // leaf centre minus anchor centre along this axis (anchor_lo is unused: offsets are relative)
      const double shift = (o + 0.5) * L - 0.5 * La;
      (void)anchor_lo;
      form_matrix(P, l, shift, Fb.data());
      eval_matrix(P, l, shift, Eb.data());
      push_complex(Ff, Fb.data(), Fb.size());
      for (int b = 0; b < nh; ++b)
        for (int j = 0; j < k; ++j) {
          const cd v = Fb[(size_t)(P.M - 1 + b) * k + j] * (b == 0 ? 1.0 : 2.0);
          Fh.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
        }
      push_complex(Ef, Eb.data(), Eb.size());
      for (int t = 0; t < k; ++t)
        for (int b = 0; b < nh; ++b) {
          const cd v = Eb[(size_t)t * n1 + P.M - 1 + b];
          Eh.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
        }
      ++nmat;
    }
    matid[key] = id;
    return id;
  };
  std::vector<int32_t> stack;
  int Kmax = 0;
  std::vector<int32_t> leaf_anchor(P.n_leaves, -1);  // anchor box of every plane-wave leaf
  auto add_block = [&](int32_t bb, int32_t anchor, int dl) {
    const Box &B = P.boxes[bb];
    const Box &A = P.boxes[anchor];
    fgt::Block blk{};
    blk.slot = A.slot;
    blk.dl = dl;
    blk.K = (1 << dl) * k;
    const int l = B.level + dl, nl = 1 << dl;
    // leaves at the cutoff level may also receive near-field terms, which run concurrently on a
    // second stream: their evaluation adds atomically into the cleared u instead of storing
    blk.flags = (l == P.lc && !P.fourier) ? 1 : 0;
    for (int a = 0; a < d; ++a) {
      const int obase = (B.c[a] << dl) - (A.c[a] << (l - A.level));
      blk.mat[a] = get_mat(l, A.level, obase, dl, 0.0);
    }
    blk.leaf0 = (int64_t)bleaves.size();
    int32_t q[3] = {0, 0, 0};
    const int tot = d == 3 ? nl * nl * nl : nl * nl;
    for (int idx = 0; idx < tot; ++idx) {
      int r = idx;
      for (int a = 0; a < d; ++a) { q[a] = (B.c[a] << dl) + (r % nl); r /= nl; }
      const int32_t lb = P.find(l, q);
      bleaves.push_back(P.boxes[lb].leaf);
      leaf_anchor[(size_t)P.boxes[lb].leaf] = anchor;
    }
    Kmax = std::max(Kmax, blk.K);
    blocks.push_back(blk);
  };
  if (hier) {
    for (int64_t i = 0; i < P.n_leaves; ++i) {
      const int32_t b = P.leaf_box[i];
      if (P.boxes[b].f) add_block(b, b, 0);
    }
  } else {
    for (int32_t a : anchors) {
      stack.assign(1, a);
      while (!stack.empty()) {
        const int32_t b = stack.back();
        stack.pop_back();
        const Box &B = P.boxes[b];
        if (B.mind == B.maxd && B.maxd <= dlcap) {
          add_block(b, a, B.maxd);
        } else {
          for (int c = nc - 1; c >= 0; --c) stack.push_back(P.children[B.child0 + c]);
        }
      }
    }
  }
  ex.n_blocks = (int64_t)blocks.size();
  ex.Kmax = Kmax;
  P.n_blocks = ex.n_blocks;

  // ---- evaluation blocks.  Without an output tree they are the form's blocks.  With one (an
  // output tree refining the source tree, Algorithm 5), an output leaf inside a source leaf B
  // evaluated by plane waves takes B's anchor: the 2^(d r) leaves of a uniform refinement of B by
  // r levels form one block of K = 2^r k (when K <= 32), any other output leaf a block of its own.
  std::vector<fgt::Block> eblocks;
  std::vector<int64_t> ebleaves;
  if (P.n_out > 0) {
    if (hier) return fail(FGT_ERR_ARG, "output trees need the fused mode");
    std::vector<std::vector<int64_t>> kids((size_t)P.n_leaves);
    for (int64_t i = 0; i < P.n_out; ++i) kids[(size_t)P.out_src[i]].push_back(i);
    for (int64_t j = 0; j < P.n_leaves; ++j) {
      const int32_t an = leaf_anchor[(size_t)j];
      if (an < 0 || kids[(size_t)j].empty()) continue;  // not evaluated by plane waves
      const Box &A = P.boxes[an];
      const Box &B = P.boxes[P.leaf_box[j]];
      const int lb = B.level;
      const std::vector<int64_t> &ks = kids[(size_t)j];
      const int r = P.out_level[(size_t)ks[0]] - lb;
      bool uniform = ((1 << r) * k <= 32) && (int64_t)ks.size() == ((int64_t)1 << (d * r));
      for (int64_t i : ks) uniform = uniform && P.out_level[(size_t)i] - lb == r;
      auto make = [&](int lt, const int32_t *cbase, int dl, const std::vector<int64_t> &leaves) {
        fgt::Block blk{};
        blk.slot = A.slot;
        blk.dl = dl;
        blk.K = (1 << dl) * k;
        blk.flags = (lb == P.lc && !P.fourier) ? 1 : 0;  // the near field also adds into these
        for (int a = 0; a < d; ++a)
          blk.mat[a] = get_mat(lt, A.level, cbase[a] - (A.c[a] << (lt - A.level)), dl, 0.0);
        blk.leaf0 = (int64_t)ebleaves.size();
        ebleaves.insert(ebleaves.end(), leaves.begin(), leaves.end());
        eblocks.push_back(blk);
      };
      if (uniform) {
        const int nl = 1 << r;
        std::vector<int64_t> order(ks.size());
        for (int64_t i : ks) {
          int idx = 0;
          for (int a = d - 1; a >= 0; --a) idx = idx * nl + (P.out_coord[(size_t)i * d + a] - (B.c[a] << r));
          order[(size_t)idx] = i;
        }
        int32_t cb[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) cb[a] = B.c[a] << r;
        make(lb + r, cb, r, order);
      } else {
        for (int64_t i : ks) make(P.out_level[(size_t)i], &P.out_coord[(size_t)i * d], 0, {i});
      }
    }
  } else {
    eblocks = blocks;
    ebleaves = bleaves;
  }

  // ---- kernel choice per block.  Form: blocks whose sigma and matrices fit in shared memory go
  // to the grouped kernel, up to 8 blocks of one anchor and one size per CTA (fewer when they
  // would not leave room for two CTAs per SM); the rest to the per-(block, m_d) kernel.
  // Evaluation: blocks with K <= 16 whose whole-block intermediates fit go to the whole-block
  // kernel; the rest to the per-(block, row) kernel.
  std::vector<fgt::Block> f1, f2, e1, e2;
  std::vector<int32_t> f2ptr(1, 0);
  int Kf1 = 0, Ke1 = 0;
  {
    const size_t rsz = P.f32() ? sizeof(float) : sizeof(double), csz = sizeof(C);
    const size_t three_per_sm = 72 * 1024;
    // 3D uses the register-tiled kernel (planes in chunks of 4), 2D the plain grouped one
    // split precision in 3D: the last contraction of the form and the first of the evaluation
    // run on the tensor cores (3xTF32) when the shapes fit the kernels' register tiles
    auto tensor_form = [&](int K) {
      return d == 3 && P.prec == FGT_PREC_SPLIT && K % 4 == 0 && 2 * ((n1 + 7) / 8 * 8) / 8 <= 14;
    };
    // the tensor-core evaluation kernel measured slower than the whole-block CUDA-core one on
    // GB300 (its stages 2-3 dominate once stage 1 is on the tensor cores), so it is off by default
    const bool tensor_eval = d == 3 && P.prec == FGT_PREC_SPLIT && nh <= 32 && P.tc_eval;
    // split precision, 3D: evaluation stages 2-3 in 3xTF32 (register tiles need K <= 32, n1 <= 56);
    // by default for blocks of K > 16 only (measured faster there, slower for K <= 16), for every
    // block with FGT_TC_EVAL4=1
    auto eval4_ok = [&](int K) {
      return d == 3 && P.prec == FGT_PREC_SPLIT && !P.tc_eval && (K > 16 || P.tc_eval4) && K <= 32 &&
             2 * ((n1 + 7) / 8) <= 14;
    };
    auto gbytes = [&](int g, int K) {
      if (tensor_form(K)) return fgt::form4_bytes(g, K, n1);
      return d == 3 ? fgt::form3_bytes(g, K, n1, rsz, csz) : fgt::form2_bytes(d, g, K, n1, nh, rsz, csz);
    };
    // split precision, 3D blocks of K > 16: one block per CTA, sigma streamed from global memory
    auto big_form = [&](int K) { return K > 16 && tensor_form(K) && fgt::form4b_bytes(K, n1) <= (size_t)smax; };
    auto gmax = [&](int K) {
      int G = 0;
      if (K > 16) return big_form(K) ? 1 : 0;  // staging sigma would leave one CTA per SM
      for (int g = 1; g <= P.tune.form_group; ++g)
        if (gbytes(g, K) <= three_per_sm) G = g;
      if (G == 0 && gbytes(1, K) <= (size_t)smax) G = 1;
      return G;
    };
    // form: groups of one anchor and one K, ordered by K so that each K gets its own launch
    // (and its own shared-memory size)
    std::vector<fgt::Block> sorted = blocks;
    std::stable_sort(sorted.begin(), sorted.end(), [](const fgt::Block &a, const fgt::Block &b) {
      return a.K != b.K ? a.K < b.K : a.slot < b.slot;
    });
    // every form stage on tcgen05 (form7_kernel) for the blocks of the sizes it takes, one block per
    // CTA: their density is packed in (J1, J2, J3) order (flags bit 2), and a block that is its
    // anchor's only one stores the slot (flags bit 1) instead of adding to it
    const bool f7_plan = P.form7 && d == 3 && P.prec == FGT_PREC_SPLIT && !hier && n1 <= 32 && nh <= 16;
    auto f7_block = [&](int K) {
      return f7_plan && (K == 16 || K == 32 || (K == 8 && P.form7_k8)) && fgt::form7_smem_bytes(K) <= (size_t)smax;
    };
    ex.sig_order = 0;
    ex.phi_stored = 0;
    size_t q = 0;
    {
      std::unordered_map<int32_t, int> per_slot;
      for (const fgt::Block &b : sorted) per_slot[b.slot]++;
      bool all_sole = true, any_f7 = false;
      for (const fgt::Block &b : sorted) all_sole = all_sole && (per_slot[b.slot] == 1 && f7_block(b.K));
      for (fgt::Block &b : blocks)
        if (f7_block(b.K)) b.flags |= 4;   // the packing order of its density
      std::vector<fgt::Block> rest;
      for (fgt::Block b : sorted) {
        if (!f7_block(b.K)) {
          rest.push_back(b);
          continue;
        }
        any_f7 = true;
        b.flags |= 4;
        const bool sole = per_slot[b.slot] == 1;
        b.flags = (b.flags & ~2) | (sole ? 2 : 0);
        if (ex.f2_ranges.empty() || ex.f2_ranges.back().K != b.K) {
          fgt::LaunchRange lr;
          lr.first = (int)f2ptr.size() - 1;
          lr.count = 0;
          lr.K = b.K;
          lr.big = b.K > 16 ? 1 : 0;
          lr.smem = fgt::form7_smem_bytes(b.K);
          lr.tensor = 7;
          ex.f2_ranges.push_back(lr);
        }
        f2.push_back(b);
        f2ptr.push_back((int32_t)f2.size());  // groups of one block
        ex.f2_ranges.back().count++;
      }
      ex.sig_order = any_f7 ? 1 : 0;
      ex.phi_stored = all_sole ? 1 : 0;
      sorted.swap(rest);  // the other blocks go to the CUDA-core forms below
    }
    while (q < sorted.size()) {
      const int K = sorted[q].K, G = gmax(K);
      if (G == 0) {
        f1.push_back(sorted[q]);
        Kf1 = std::max(Kf1, K);
        ++q;
        continue;
      }
      const int first_group = (int)f2ptr.size() - 1;
      while (q < sorted.size() && sorted[q].K == K) {
        const int32_t slot = sorted[q].slot;
        int n = 0;
        while (q < sorted.size() && sorted[q].K == K && sorted[q].slot == slot && n < G) {
          f2.push_back(sorted[q]);
          ++q;
          ++n;
        }
        f2ptr.push_back((int32_t)f2.size());
      }
      fgt::LaunchRange lr;
      lr.first = first_group;
      lr.count = (int)f2ptr.size() - 1 - first_group;
      lr.K = K;
      lr.big = K > 16 ? 1 : 0;
      lr.smem = lr.big ? fgt::form4b_bytes(K, n1) : gbytes(G, K);
      lr.tensor = (tensor_form(K) || (ex.tc64 && d == 3)) ? 1 : 0;
      ex.f2_ranges.push_back(lr);
    }
    // evaluation: whole-block kernel for K <= 16 when it fits, one launch per K; in split
    // precision (3D) larger blocks too, a few rows per CTA
    // rows per CTA (split precision, 3D): by default 8 for K = 16 and 4 for larger blocks, which
    // measured fastest on GB300 (more resident CTAs outweigh reading the anchor's expansion two or
    // more times)
    auto norm_rows = [](int r) { return r <= 4 ? 4 : r <= 8 ? 8 : 16; };  // the kernel's instantiations
    const int rows16 = norm_rows(P.tune.eval_rows16), rows32 = norm_rows(P.tune.eval_rows_large);
    // 3D: the evaluation with the half-range axis last (fewer products), rows I1 per CTA as many
    // as keep its shared memory within e5_budget
    const size_t e5_budget = P.f32() ? 80 * 1024 : 112 * 1024;
    auto e5_rows = [&](int K) {
      for (int rc : {16, 8, 4, 2, 1})
        if (rc <= K && fgt::eval5_bytes(K, n1, nh, csz, rc) <= e5_budget) return rc;
      return fgt::eval5_bytes(K, n1, nh, csz, 1) <= (size_t)smax ? 1 : 0;
    };
    const bool use_e5 = d == 3 && P.eval5 && !P.tc_eval && !ex.tc64;
    std::vector<fgt::Block> esorted = eblocks;
    std::stable_sort(esorted.begin(), esorted.end(), [](const fgt::Block &a, const fgt::Block &b) {
      return a.K != b.K ? a.K < b.K : a.slot < b.slot;
    });
    // every evaluation stage on tcgen05 (eval7_kernel): it reads the incoming expansions in a padded
    // layout of its own, so it takes all blocks of the plan or none
    bool use_e7 = P.eval7 && d == 3 && P.prec == FGT_PREC_SPLIT && !hier && !P.fourier && k % 2 == 0 &&
                  n1 <= fgt::eval7_pitch() && !P.tc_eval && !P.tc_eval4 && !P.tc_eval6 && !P.eval5 &&
                  !esorted.empty();
    for (const fgt::Block &b : esorted)
      use_e7 = use_e7 && (b.K == 8 || b.K == 16 || b.K == 32) && fgt::eval7_smem_bytes(b.K) <= (size_t)smax;
    ex.psi_pitch = use_e7 ? fgt::eval7_pitch() : 0;
    for (const fgt::Block &b : esorted) {
      if (use_e7) {
        if (ex.e2_ranges.empty() || ex.e2_ranges.back().K != b.K) {
          fgt::LaunchRange lr;
          lr.first = (int)e2.size();
          lr.count = 0;
          lr.K = b.K;
          // rows per CTA of the CUDA-core kernel that stands in where the padded layout is off
          lr.rows = b.K <= 8 ? 8 : b.K <= 16 ? rows16 : rows32;
          lr.smem = fgt::eval7_smem_bytes(b.K);
          lr.tensor = 7;
          ex.e2_ranges.push_back(lr);
        }
        e2.push_back(b);
        ex.e2_ranges.back().count++;
        continue;
      }
      if (use_e5 && e5_rows(b.K) > 0) {
        const int rc = e5_rows(b.K);
        if (ex.e2_ranges.empty() || ex.e2_ranges.back().K != b.K) {
          fgt::LaunchRange lr;
          lr.first = (int)e2.size();
          lr.count = 0;
          lr.K = b.K;
          lr.rows = rc;
          lr.smem = fgt::eval5_bytes(b.K, n1, nh, csz, rc);
          lr.tensor = 3;
          ex.e2_ranges.push_back(lr);
        }
        e2.push_back(b);
        ex.e2_ranges.back().count++;
        continue;
      }
      const bool chunked = b.K > 16 && d == 3 && (P.prec == FGT_PREC_SPLIT || ex.tc64);
      const int rows = b.K <= 8 ? 8 : b.K <= 16 ? (P.prec == FGT_PREC_SPLIT && d == 3 ? rows16 : 16) : rows32;
      // split precision, 3D, K <= 16: stage 1 on tcgen05 when its accumulators fit tensor memory;
      // shared memory padded so that the CTAs an SM can hold never ask for more than its 512 columns
      const int tc6_cols = fgt::eval6_tmem_cols(n1, rows);
      if (d == 3 && P.prec == FGT_PREC_SPLIT && P.tc_eval6 && !P.tc_eval && !P.tc_eval4 && b.K <= 16 &&
          tc6_cols > 0 && fgt::eval6_kpad(nh) <= fgt::kEval6MaxKp2) {
        size_t sm6 = fgt::eval6_bytes(b.K, n1, nh, rows);
        // CTAs an SM holds: 228 KB of shared memory, 1 KB reserved per CTA, at most 8 of 256 threads
        auto ctas = [](size_t b) { return std::min<size_t>(8, 233472 / (b + 1024)); };
        while (ctas(sm6) * (size_t)tc6_cols > 512) sm6 += 1024;
        if (sm6 <= (size_t)smax) {
          if (ex.e2_ranges.empty() || ex.e2_ranges.back().K != b.K) {
            fgt::LaunchRange lr;
            lr.first = (int)e2.size();
            lr.count = 0;
            lr.K = b.K;
            lr.rows = rows;
            lr.smem = sm6;
            lr.tensor = 4;
            lr.tmem_cols = tc6_cols;
            ex.e2_ranges.push_back(lr);
          }
          e2.push_back(b);
          ex.e2_ranges.back().count++;
          continue;
        }
      }
      const size_t eb = (tensor_eval && !chunked) ? fgt::eval3_bytes(b.K, n1, nh)
                                                  : fgt::eval2_bytes(d, b.K, n1, nh, csz, rows);
      if ((b.K <= 16 || chunked) && eb <= (size_t)smax) {
        if (ex.e2_ranges.empty() || ex.e2_ranges.back().K != b.K) {
          fgt::LaunchRange lr;
          lr.first = (int)e2.size();
          lr.count = 0;
          lr.K = b.K;
          lr.rows = rows;
          lr.smem = eb;
          lr.tensor = ((tensor_eval && !chunked) || (ex.tc64 && d == 3)) ? 1 : 0;
          if (eval4_ok(b.K)) lr.tensor = 2;  // stages 2-3 of the evaluation on the tensor cores
          ex.e2_ranges.push_back(lr);
        }
        e2.push_back(b);
        ex.e2_ranges.back().count++;
      } else {
        e1.push_back(b);
        Ke1 = std::max(Ke1, b.K);
      }
    }
  }
  ex.n_f1 = (int64_t)f1.size();
  ex.Kmax_f1 = Kf1;
  ex.n_f2_groups = (int64_t)f2ptr.size() - 1;
  ex.n_e1 = (int64_t)e1.size();
  ex.Kmax_e1 = Ke1;
  ex.n_e2 = (int64_t)e2.size();

  // ---- FP64 on the BF16 tensor cores by exact slicing (precision FP64_TC, 3D, fused mode): the
  // form's and the evaluation's contractions as six stages of the sliced-stage kernel.  Each block's
  // 1D matrix of a stage, in the real form of its complex contraction, is cut here once into six
  // balanced 8-bit digits per entry against its column's largest exponent (exact: a 47-bit rounding
  // of each entry, then integer digits), laid out as the kernel's bulk copies read it: per column
  // part and 16-deep step, six BF16 planes in the K-major core-matrix layout.  The block lists above
  // stay, for the allocation-free call.
  std::vector<fgt::OzJob> ozjobs[6], ozsjobs[6];
  std::vector<fgt::OzGroup> ozgroups;
  std::vector<unsigned char> oztab;
  std::vector<int32_t> ozexp;
  int64_t oz_scr = 0;  // doubles per scratch array
  int64_t oz_dig = 0, oz_rexp = 0;  // bytes of the digit planes, row exponents of the largest stage
  ex.oz = 0;
  ex.oz_sole = 0;
  if constexpr (std::is_same<C, double2>::value) {
    if (P.prec == FGT_PREC_FP64_TC && P.ozaki && d == 3 && !hier && !P.fourier && n1 <= 80 && !blocks.empty()) {
      ex.oz = 1;
      std::map<std::tuple<int, int, int>, std::pair<int64_t, int32_t>> cls;
      std::vector<double> Bm;
      // the digit planes of Bm (dm.Q x dm.N, row-major) in the layout the products kernel copies:
      // per column part and 16-deep step, six BF16 planes of Np rows in the K-major core-matrix layout
      auto slice_bm = [&](const fgt::OzDims &dm) -> std::pair<int64_t, int32_t> {
        auto B = [&](int q, int n) -> double & { return Bm[(size_t)q * dm.N + n]; };
        const int64_t boff = (int64_t)oztab.size();
        const int32_t eoff = (int32_t)ozexp.size();
        const size_t bbytes = (size_t)fgt::kOzSlices * dm.Np * 32;
        oztab.resize(oztab.size() + (size_t)dm.P * dm.nks * bbytes, 0);
        for (int pt = 0; pt < dm.P; ++pt)
          for (int nl = 0; nl < dm.Np; ++nl) {
            const int c = pt * dm.Nc + nl;
            const bool valid = nl < dm.Nc && c < dm.N;
            double mx = 0.0;
            if (valid)
              for (int q = 0; q < dm.Q; ++q) mx = std::max(mx, std::fabs(B(q, c)));
            int f = 0;
            if (mx > 0) std::frexp(mx, &f);  // |B(q, c)| < 2^f
            ozexp.push_back(f);
            if (mx == 0) continue;
            for (int q = 0; q < dm.Q; ++q) {
              long long v = std::llrint(std::ldexp(B(q, c), 47 - f));  // |v| <= 2^47, exact scaling
              int dg[fgt::kOzSlices];
              for (int sl = fgt::kOzSlices - 1; sl >= 1; --sl) {
                const int lo = (int)((v + 128) & 255) - 128;
                dg[sl] = lo;
                v = (v - lo) / 256;
              }
              dg[0] = (int)v;
              const int ks = q / 16, kk = q % 16;
              for (int sl = 0; sl < fgt::kOzSlices; ++sl) {
                const float fv = (float)dg[sl];
                uint32_t bits;
                std::memcpy(&bits, &fv, 4);
                const uint16_t h = (uint16_t)(bits >> 16);  // exact: |digit| <= 128
                const size_t off = (size_t)boff + ((size_t)(pt * dm.nks + ks) * fgt::kOzSlices + sl) * dm.Np * 32 +
                                   (size_t)(nl >> 3) * 256 + (size_t)(kk >> 3) * 128 + (size_t)(nl & 7) * 16 +
                                   (size_t)(kk & 7) * 2;
                std::memcpy(&oztab[off], &h, 2);
              }
            }
          }
        return {boff, eoff};
      };
      auto table = [&](int kind, int K, int mat) -> std::pair<int64_t, int32_t> {
        const auto key = std::make_tuple(kind, K, mat);
        auto it = cls.find(key);
        if (it != cls.end()) return it->second;
        const fgt::OzDims dm = fgt::oz_dims(kind, K, n1, nh);
        Bm.assign((size_t)dm.Q * dm.N, 0.0);
        auto B = [&](int q, int n) -> double & { return Bm[(size_t)q * dm.N + n]; };
        if (kind == 0) {  // x3, half range: q = J3, n = (m3, c); sigma is real
          for (int J = 0; J < K; ++J)
            for (int m = 0; m < nh; ++m) {
              const C f = Fh[((size_t)(mat + J / k) * nh + m) * k + J % k];
              B(J, 2 * m) = f.x;
              B(J, 2 * m + 1) = f.y;
            }
        } else if (kind <= 2) {  // x2 / x1: q = (c, J), n = (m, c')
          for (int J = 0; J < K; ++J)
            for (int m = 0; m < n1; ++m) {
              const C f = Ff[((size_t)(mat + J / k) * n1 + m) * k + J % k];
              B(J, 2 * m) = f.x;
              B(K + J, 2 * m) = -f.y;
              B(J, 2 * m + 1) = f.y;
              B(K + J, 2 * m + 1) = f.x;
            }
        } else if (kind <= 4) {  // m1: q = (m, c), n = (c', I); m2: q = (c, m), n = (c', I)
          for (int I = 0; I < K; ++I)
            for (int m = 0; m < n1; ++m) {
              const C e = Ef[((size_t)(mat + I / k) * k + I % k) * n1 + m];
              const int q0 = kind == 3 ? 2 * m : m, q1 = kind == 3 ? 2 * m + 1 : n1 + m;
              B(q0, I) = e.x;
              B(q1, I) = -e.y;
              B(q0, K + I) = e.y;
              B(q1, K + I) = e.x;
            }
        } else {  // m3, half range, real part: q = (c, m3), n = I3
          for (int I = 0; I < K; ++I)
            for (int m = 0; m < nh; ++m) {
              const C e = Eh[((size_t)(mat + I / k) * k + I % k) * nh + m];
              B(m, I) = e.x;
              B(nh + m, I) = -e.y;
            }
        }
        const auto r = slice_bm(dm);
        cls[key] = r;
        return r;
      };
      int64_t dig_at[6] = {0, 0, 0, 0, 0, 0}, rexp_at[6] = {0, 0, 0, 0, 0, 0};
      // the evaluation's first stage reads the anchor's incoming expansion, the same for every block of
      // the anchor: it is sliced once per anchor, and each block's products read those digit planes
      std::unordered_map<int32_t, std::pair<int64_t, int32_t>> slot_digits;
      auto add_jobs = [&](int kind, int32_t bi, const fgt::Block &B, int64_t scr, int flags) {
        const int mat = B.mat[(kind == 0 || kind == 5) ? 2 : (kind == 1 || kind == 4) ? 1 : 0];
        const auto tb = table(kind, B.K, mat);
        const fgt::OzDims dm = fgt::oz_dims(kind, B.K, n1, nh);
        const int ntile = (dm.R + 127) / 128;
        const int64_t tile_bytes = (int64_t)dm.nks * fgt::kOzSlices * 128 * 16 * 2;
        int64_t a0 = dig_at[kind];
        int32_t r0 = (int32_t)rexp_at[kind];
        bool slice = true;
        if (kind == 3) {
          auto it = slot_digits.find(B.slot);
          if (it != slot_digits.end()) {
            a0 = it->second.first;
            r0 = it->second.second;
            slice = false;
          } else {
            slot_digits[B.slot] = {a0, r0};
          }
        }
        for (int t = 0; t < ntile; ++t) {
          fgt::OzJob j{};
          j.blk = bi;
          j.tile = (int16_t)t;
          j.scr = scr;
          j.aoff = a0 + t * tile_bytes;
          j.roff = r0 + 128 * t;
          j.flags = flags;
          j.nks = (int16_t)dm.nks;
          j.np = (int16_t)dm.Np;
          if (slice) ozsjobs[kind].push_back(j);  // slicing: part 0 stands for the tile
          for (int pt = 0; pt < dm.P; ++pt) {
            j.part = (int16_t)pt;
            j.boff = tb.first + (int64_t)pt * dm.nks * fgt::kOzSlices * dm.Np * 32;
            j.eoff = tb.second + pt * dm.Np;
            ozjobs[kind].push_back(j);
          }
        }
        if (slice) {
          dig_at[kind] += ntile * tile_bytes;
          rexp_at[kind] += 128 * ntile;
        }
      };
      // per-block intermediates: the form's and the evaluation's stages reuse the same two arrays
      bool all_sole = true;
      int64_t sf = 0, se = 0;
      // stage 2 (x1, into the slot) by groups of the anchor's consecutive blocks, their contractions
      // concatenated up to 160 (the exactness bound) and kOzGroupMax members
      std::vector<fgt::OzGroup> groups;
      std::map<std::vector<int32_t>, std::pair<int64_t, int32_t>> gcls;
      auto group_table = [&](const fgt::OzGroup &g, const std::vector<int32_t> &mats) {
        std::vector<int32_t> key;
        for (int m = 0; m < g.n; ++m) {
          key.push_back(g.K[m]);
          key.push_back(mats[m]);
        }
        auto it = gcls.find(key);
        if (it != gcls.end()) return it->second;
        const fgt::OzDims dm = fgt::oz_dims_group(n1, nh, g.q0[g.n]);
        Bm.assign((size_t)dm.Q * dm.N, 0.0);
        auto B = [&](int q, int n) -> double & { return Bm[(size_t)q * dm.N + n]; };
        for (int m = 0; m < g.n; ++m) {  // member m: rows q0 + (c, J1) as in its own stage-2 matrix
          const int K = g.K[m], q0 = g.q0[m], mat = mats[m];
          for (int J = 0; J < K; ++J)
            for (int mm = 0; mm < n1; ++mm) {
              const C f = Ff[((size_t)(mat + J / k) * n1 + mm) * k + J % k];
              B(q0 + J, 2 * mm) = f.x;
              B(q0 + K + J, 2 * mm) = -f.y;
              B(q0 + J, 2 * mm + 1) = f.y;
              B(q0 + K + J, 2 * mm + 1) = f.x;
            }
        }
        const auto r = slice_bm(dm);
        gcls[key] = r;
        return r;
      };
      std::vector<int64_t> block_scr(blocks.size());
      for (size_t b = 0; b < blocks.size(); ++b) {
        const fgt::Block &B = blocks[b];
        const int64_t K = B.K;
        block_scr[b] = sf;
        for (int kind = 0; kind < 2; ++kind) add_jobs(kind, (int32_t)b, B, sf, 0);
        sf += std::max<int64_t>(2 * nh * K * K, 2 * (int64_t)n1 * nh * K);
      }
      std::vector<std::vector<int32_t>> gmats;
      for (size_t b = 0; b < blocks.size();) {
        fgt::OzGroup g{};
        g.slot = blocks[b].slot;
        std::vector<int32_t> mats;
        while (b < blocks.size() && blocks[b].slot == g.slot && g.n < fgt::kOzGroupMax &&
               g.q0[g.n] + 2 * blocks[b].K <= 160) {
          g.K[g.n] = blocks[b].K;
          g.blk[g.n] = (int32_t)b;
          g.scr[g.n] = block_scr[b];
          g.q0[g.n + 1] = g.q0[g.n] + 2 * blocks[b].K;
          mats.push_back(blocks[b].mat[0]);
          ++g.n;
          ++b;
        }
        groups.push_back(g);
        gmats.push_back(mats);
      }
      std::unordered_map<int32_t, int> groups_per_slot;
      for (const fgt::OzGroup &g : groups) groups_per_slot[g.slot]++;
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        const fgt::OzGroup &g = groups[gi];
        const bool sole = groups_per_slot[g.slot] == 1;
        all_sole = all_sole && sole;
        const auto tb = group_table(g, gmats[gi]);
        const fgt::OzDims dm = fgt::oz_dims_group(n1, nh, g.q0[g.n]);
        const int ntile = (dm.R + 127) / 128;
        const int64_t tile_bytes = (int64_t)dm.nks * fgt::kOzSlices * 128 * 16 * 2;
        for (int t = 0; t < ntile; ++t) {
          fgt::OzJob j{};
          j.blk = (int32_t)gi;
          j.tile = (int16_t)t;
          j.aoff = dig_at[2] + t * tile_bytes;
          j.roff = (int32_t)rexp_at[2] + 128 * t;
          j.flags = sole ? 0 : 1;
          j.nks = (int16_t)dm.nks;
          j.np = (int16_t)dm.Np;
          ozsjobs[2].push_back(j);
          for (int pt = 0; pt < dm.P; ++pt) {
            j.part = (int16_t)pt;
            j.boff = tb.first + (int64_t)pt * dm.nks * fgt::kOzSlices * dm.Np * 32;
            j.eoff = tb.second + pt * dm.Np;
            ozjobs[2].push_back(j);
          }
        }
        dig_at[2] += ntile * tile_bytes;
        rexp_at[2] += 128 * ntile;
      }
      for (size_t b = 0; b < eblocks.size(); ++b) {
        const fgt::Block &B = eblocks[b];
        const int64_t K = B.K;
        for (int kind = 3; kind < 6; ++kind) add_jobs(kind, (int32_t)b, B, se, kind == 5 ? (B.flags & 1) : 0);
        se += std::max<int64_t>(2 * K * nh * n1, 2 * K * K * nh);
      }
      oz_scr = std::max(sf, se);
      ex.oz_sole = all_sole ? 1 : 0;
      ozgroups = groups;
      for (int kind = 0; kind < 6; ++kind) {
        ex.oz_njobs[kind] = (int64_t)ozjobs[kind].size();
        ex.oz_nsjobs[kind] = (int64_t)ozsjobs[kind].size();
        oz_dig = std::max(oz_dig, dig_at[kind]);
        oz_rexp = std::max(oz_rexp, rexp_at[kind]);
      }
    }
  }

  // ---- out->in gather at the cutoff level (P-list)
  std::vector<int32_t> gdst;
  std::vector<int64_t> gptr(1, 0);
  std::vector<fgt::GatherSrc> gsrc;
  const bool per = P.bc == FGT_BC_PERIODIC;
  int noff = 1;
  for (int a = 0; a < d; ++a) noff *= 3;
  if (!P.fourier) {
    const int nb = 1 << P.lc;
    for (int32_t T : anchors) {
      const Box &Tb = P.boxes[T];
      for (int oc = 0; oc < noff; ++oc) {
        int32_t q[3] = {0, 0, 0};
        bool ok = true;
        int code = 0, mul = 1;
        for (int a = 0, r = oc; a < d; ++a, r /= 3) {
          const int o = r % 3 - 1;
          int v = Tb.c[a] + o;
          if (v < 0 || v >= nb) {
            if (!per) { ok = false; break; }
            v = (v + nb) % nb;
          }
          q[a] = v;
          code += (o + 1) * mul;
          mul *= 3;
        }
        if (!ok) continue;
        const int32_t S = P.find(P.lc, q);
        if (S < 0 || !P.boxes[S].f) continue;
        gsrc.push_back(fgt::GatherSrc{P.boxes[S].slot, code});
      }
      gdst.push_back(Tb.slot);
      gptr.push_back((int64_t)gsrc.size());
    }
  }
  ex.n_gather = (int64_t)gdst.size();
  P.n_gather_pairs = (int64_t)gsrc.size();
  // the same gather in separable form (all precisions; FP64 with FGT_GATHER2=0 keeps the other),
  // runs of kSegW target boxes along x_1, each with the 3^(d-1) neighbouring source lines (one
  // launch item per run)
  std::vector<fgt::GatherSeg> gsegs;
  ex.seg_w = 0;
  if ((P.prec == FGT_PREC_SPLIT || P.gather2_fp64) && !P.fourier && !anchors.empty()) {
    const int nb = 1 << P.lc, sw = std::min(fgt::kSegW, nb);
    ex.seg_w = sw;
    std::map<std::array<int32_t, 3>, size_t> seg_of;
    auto slot_at = [&](int32_t x, int32_t y, int32_t z) -> int32_t {
      int32_t q[3] = {x, y, z};
      for (int a = 0; a < d; ++a) {
        if (q[a] < 0 || q[a] >= nb) {
          if (!per) return -1;
          q[a] = (q[a] % nb + nb) % nb;
        }
      }
      const int32_t S = P.find(P.lc, q);
      return (S >= 0 && P.boxes[S].f) ? P.boxes[S].slot : -1;
    };
    for (int32_t T : anchors) {
      const Box &Tb = P.boxes[T];
      const int32_t x0 = Tb.c[0] / sw * sw, y = Tb.c[1], z = d == 3 ? Tb.c[2] : 0;
      const std::array<int32_t, 3> key{x0, y, z};
      auto it = seg_of.find(key);
      if (it == seg_of.end()) {
        fgt::GatherSeg g;
        for (int t = 0; t < fgt::kSegW; ++t) g.tgt[t] = -1;
        for (int l = 0; l < 9; ++l) {
          // 2D uses lines 0..2 (o_2 = l - 1) only
          const int o2 = l % 3 - 1, o3 = d == 3 ? l / 3 - 1 : 0;
          for (int i = 0; i < fgt::kSegW + 2; ++i) {
            // only the sw + 2 boxes around a run of sw targets are ever read
            g.src[l][i] = (i < sw + 2 && (d == 3 || l < 3)) ? slot_at(x0 - 1 + i, y + o2, z + o3) : -1;
          }
        }
        it = seg_of.emplace(key, gsegs.size()).first;
        gsegs.push_back(g);
      }
      gsegs[it->second].tgt[Tb.c[0] - x0] = Tb.slot;
    }
  }
  ex.n_gather_segs = (int64_t)gsegs.size();
  // FP64 expansions, every box of the cutoff level an anchor (3D, 4 or 8 boxes a side): the stencil
  // form of the gather over the whole grid (measured 2.0x faster than the run form on the
  // 16.8M-point periodic workload at tol 1e-10, 1.6x on the adaptive one; in FP32 the run form
  // measured faster, 0.064 against 0.075 ms); FGT_GATHER3=0 keeps the run form
  std::vector<int32_t> ggrid;
  ex.grid_nb = 0;
  ex.grid_periodic = per ? 1 : 0;
  // FP64-TC plans also take the cutoff grids with empty boxes (4, 8 or 16 boxes a side): the line
  // stencil over the whole grid reads every slot once per mode (on full grids it measured slower
  // than gather3: 0.304 against 0.255 ms on the 16.8M-point periodic workload at tol 1e-10)
  ex.grid_lines = 0;
  const bool lines_ok = P.prec == FGT_PREC_FP64_TC && (P.lc >= 2 && P.lc <= 4);
  if (d == 3 && !P.fourier && P.gather3 && !P.f32() && !hier && ((P.lc == 2 || P.lc == 3) || lines_ok) &&
      !anchors.empty()) {
    const int nb = 1 << P.lc;
    ggrid.assign((size_t)nb * nb * nb, -1);
    bool full = (int64_t)anchors.size() == (int64_t)nb * nb * nb;
    for (int32_t T : anchors) {
      const Box &Tb = P.boxes[T];
      ggrid[((size_t)Tb.c[2] * nb + Tb.c[1]) * nb + Tb.c[0]] = Tb.slot;
    }
    for (int32_t v : ggrid) full = full && v >= 0;
    if (full && P.lc <= 3) {
      ex.grid_nb = nb;
    } else if (lines_ok) {
      ex.grid_nb = nb;
      ex.grid_lines = 1;
    } else {
      ggrid.clear();
    }
  }
  // phase vectors of T_out->in: S = T + o (box units) gives c_T - c_S = -o L_c
  std::vector<C> Pf, Ph;
  {
    const double Lc = std::ldexp(1.0, -P.lc);
    for (int o = -1; o <= 1; ++o)
      for (int a = 0; a < n1; ++a) {
        const cd v = std::polar(1.0, -P.kappa * (a - (P.M - 1)) * o * Lc);
        Pf.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
      }
    for (int o = -1; o <= 1; ++o)
      for (int b = 0; b < nh; ++b) {
        const cd v = std::polar(1.0, -P.kappa * b * o * Lc);
        Ph.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
      }
  }

  // the stencil gather's symmetric form needs the offset-0 factors to be 1 and the +1 factors the
  // conjugates of the -1 ones, exactly (true of polar(1, +-theta), checked rather than assumed)
  ex.gather_sym = 1;
  for (int a = 0; a < n1; ++a)
    ex.gather_sym &= (Pf[(size_t)n1 + a].x == 1 && Pf[(size_t)n1 + a].y == 0 && Pf[(size_t)2 * n1 + a].x == Pf[a].x &&
                      Pf[(size_t)2 * n1 + a].y == -Pf[a].y) ? 1 : 0;
  for (int b = 0; b < nh; ++b)
    ex.gather_sym &= (Ph[(size_t)nh + b].x == 1 && Ph[(size_t)nh + b].y == 0 && Ph[(size_t)2 * nh + b].x == Ph[b].x &&
                      Ph[(size_t)2 * nh + b].y == -Ph[b].y) ? 1 : 0;

  // ---- hierarchical merge / push lists and phases
  struct StepHost { std::vector<fgt::TreeShift> items; std::vector<C> qf, qh; };
  std::vector<StepHost> merge_h, push_h;
  if (hier) {
    auto phases = [&](int child_level, double sign, std::vector<C> &qf, std::vector<C> &qh) {
      const double Lch = std::ldexp(1.0, -child_level);
      for (int bit = 0; bit < 2; ++bit)
        for (int a = 0; a < n1; ++a) {
          const cd v = std::polar(1.0, sign * P.kappa * (a - (P.M - 1)) * (bit - 0.5) * Lch);
          qf.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
        }
      for (int bit = 0; bit < 2; ++bit)
        for (int b = 0; b < nh; ++b) {
          const cd v = std::polar(1.0, sign * P.kappa * b * (bit - 0.5) * Lch);
          qh.push_back(C{(decltype(C::x))v.real(), (decltype(C::x))v.imag()});
        }
    };
    auto items_at = [&](int l) {
      std::vector<fgt::TreeShift> v;
      for (int32_t b : P.by_level[l]) {
        const Box &B = P.boxes[b];
        if (B.leaf >= 0 || !B.f) continue;
        fgt::TreeShift it{};
        it.parent = B.slot;
        for (int c = 0; c < nc; ++c) it.child[c] = P.boxes[P.children[B.child0 + c]].slot;
        v.push_back(it);
      }
      return v;
    };
    for (int l = P.lmax - 1; l >= P.lc; --l) {
      StepHost s;
      s.items = items_at(l);
      phases(l + 1, -1.0, s.qf, s.qh);  // T_c->p = exp(-i k (c_child - c_parent))
      merge_h.push_back(std::move(s));
    }
    for (int l = P.lc; l <= P.lmax - 1; ++l) {
      StepHost s;
      s.items = items_at(l);
      phases(l + 1, +1.0, s.qf, s.qh);  // T_p->c = exp(+i k (c_child - c_parent))
      push_h.push_back(std::move(s));
    }
  }

  // ---- near field (D-list)
  std::vector<int64_t> ntgt, nptr(1, 0);
  std::vector<int32_t> nflags;
  std::vector<fgt::NearSrc> nsrc;
  std::vector<double> ntab;
  if (!P.fourier) {
    const int ltab = std::min(P.lc, P.lmax);
    std::vector<char> level_used(ltab + 1, 0);
    struct Cand { int32_t box; int n[3]; };
    std::vector<Cand> cands;
    for (int64_t i = 0; i < P.n_leaves; ++i) {
      const int32_t T = P.leaf_box[i];
      const Box &Tb = P.boxes[T];
      if (Tb.level > P.lc) continue;
      const int l = Tb.level, nb = 1 << l;
      cands.clear();
      for (int oc = 0; oc < noff; ++oc) {
        int o[3] = {0, 0, 0}, q[3] = {0, 0, 0}, img[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0, r = oc; a < d; ++a, r /= 3) {
          o[a] = r % 3 - 1;
          int v = Tb.c[a] + o[a];
          if (v < 0 || v >= nb) {
            if (!per) { ok = false; break; }
            img[a] = v < 0 ? -1 : 1;
            v -= img[a] * nb;
          }
          q[a] = v;
        }
        if (!ok) continue;
        const int32_t N = P.find(l, q);
        auto add = [&](int32_t s) {
          for (const Cand &c : cands)
            if (c.box == s && c.n[0] == img[0] && c.n[1] == img[1] && c.n[2] == img[2]) return;
          cands.push_back(Cand{s, {img[0], img[1], img[2]}});
        };
        if (N >= 0) {
          const Box &Nb = P.boxes[N];
          if (Nb.leaf >= 0) {
            add(N);
          } else if (l < P.lc) {
            for (int c = 0; c < nc; ++c) {
              bool touch = true;
              for (int a = 0; a < d; ++a) {
                const int bit = (c >> a) & 1;
                if ((o[a] == 1 && bit != 0) || (o[a] == -1 && bit != 1)) touch = false;
              }
              if (touch) add(P.children[Nb.child0 + c]);
            }
          }
        } else {
          int32_t pq[3] = {0, 0, 0};
          for (int a = 0; a < d; ++a) pq[a] = q[a] >> 1;
          const int32_t cb = (l >= 1) ? P.find(l - 1, pq) : -1;
          if (cb < 0) return fail(FGT_ERR_TREE, "internal: missing coarse neighbour");
          add(cb);
        }
      }
      const size_t before = nsrc.size();
      for (const Cand &c : cands) {
        const Box &Sb = P.boxes[c.box];
        if (Tb.level == P.lc && Sb.level == P.lc && Tb.f && Sb.f) continue;  // plane-wave pair
        fgt::NearSrc ns{};
        ns.leaf = Sb.leaf;
        const double Ls = std::ldexp(1.0, -Sb.level), Lt = std::ldexp(1.0, -Tb.level);
        for (int a = 0; a < d; ++a) {
          const double ct = -0.5 + (Tb.c[a] + 0.5) * Lt;
          const double cs = -0.5 + (Sb.c[a] + 0.5) * Ls + c.n[a];
          const int o4 = (int)std::lround(4.0 * (ct - cs) / Ls);
          const int kind = near_kind(Tb.level - Sb.level, o4);
          if (kind < 0) return fail(FGT_ERR_TREE, "internal: unexpected neighbour geometry");
          ns.tab[a] = Sb.level * fgt::kNearTypes + kind;
        }
        level_used[Sb.level] = 1;
        nsrc.push_back(ns);
      }
      if (nsrc.size() > before) {
        ntgt.push_back(i);
        nflags.push_back(Tb.f ? 1 : 0);
        nptr.push_back((int64_t)nsrc.size());
      }
    }
    ntab.assign((size_t)(ltab + 1) * fgt::kNearTypes * k * k, 0.0);
    for (int l = 0; l <= ltab; ++l) {
      if (!level_used[l]) continue;
      for (int kind = 0; kind < fgt::kNearTypes; ++kind) {
        int o4, ldiff;
        double ratio;
        kind_geometry(kind, o4, ldiff, ratio);
        near_table(P, l, 0.5 * o4, ratio, ntab.data() + ((size_t)l * fgt::kNearTypes + kind) * k * k);
      }
    }
  }
  ex.n_near = (int64_t)ntgt.size();
  // The pairs to apply: every D-list pair of the source tree, or with an output tree, each
  // output leaf paired with the D-list sources of the source leaf containing it, through tables for
  // the output leaf's own nodes (same source box, target interval of the finer box; Algorithm 5).
  const size_t kk2 = (size_t)k * k;
  size_t n_std_tables = ntab.size() / std::max<size_t>(kk2, 1);
  std::vector<int> tab_ls(n_std_tables);
  for (size_t t = 0; t < n_std_tables; ++t) tab_ls[t] = (int)(t / fgt::kNearTypes);
  std::vector<fgt::NearPair> raw;
  if (P.n_out == 0) {
    for (size_t i = 0; i < ntgt.size(); ++i)
      for (int64_t q = nptr[i]; q < nptr[i + 1]; ++q) {
        fgt::NearPair pr{};
        pr.tgt = ntgt[i];
        pr.src = nsrc[q].leaf;
        for (int a = 0; a < 3; ++a) pr.tab[a] = nsrc[q].tab[a];
        raw.push_back(pr);
      }
  } else {
    std::vector<int64_t> row_of((size_t)P.n_leaves, -1);
    for (size_t i = 0; i < ntgt.size(); ++i) row_of[(size_t)ntgt[i]] = (int64_t)i;
    std::map<std::tuple<int, int, int64_t>, int32_t> extra;  // (source level, target level, offset) -> table
    for (int64_t ti = 0; ti < P.n_out; ++ti) {
      const int64_t j = P.out_src[(size_t)ti];
      const int64_t i = row_of[(size_t)j];
      if (i < 0) continue;
      const int lt = P.out_level[(size_t)ti], lb = P.leaf_level[(size_t)j];
      for (int64_t q = nptr[(size_t)i]; q < nptr[(size_t)i + 1]; ++q) {
        fgt::NearPair pr{};
        pr.tgt = ti;
        pr.src = nsrc[q].leaf;
        for (int a = 0; a < 3; ++a) pr.tab[a] = nsrc[q].tab[a];
        if (lt != lb) {
          for (int a = 0; a < d; ++a) {
            const int ls = nsrc[q].tab[a] / fgt::kNearTypes, kind = nsrc[q].tab[a] % fgt::kNearTypes;
            int o4, ldiff;
            double ratio;
            kind_geometry(kind, o4, ldiff, ratio);
            const double Ls = std::ldexp(1.0, -ls), Lt = std::ldexp(1.0, -lt), Lb = std::ldexp(1.0, -lb);
            const double cb = -0.5 + (P.leaf_coord[(size_t)j * d + a] + 0.5) * Lb;
            const double ct = -0.5 + (P.out_coord[(size_t)ti * d + a] + 0.5) * Lt;
            const double off = (ct - cb) + 0.25 * o4 * Ls;  // target centre minus source centre (image)
            const int64_t key = std::llround(off / (0.25 * std::min(Lt, Ls)));
            auto it = extra.find({ls, lt, key});
            int32_t id;
            if (it == extra.end()) {
              id = (int32_t)(ntab.size() / kk2);
              ntab.resize(ntab.size() + kk2);
              near_table(P, ls, off / (0.5 * Ls), Lt / Ls, ntab.data() + (size_t)id * kk2);
              tab_ls.push_back(ls);
              extra.emplace(std::make_tuple(ls, lt, key), id);
            } else {
              id = it->second;
            }
            pr.tab[a] = id;
          }
        }
        raw.push_back(pr);
      }
    }
  }
  // Bands of the near-field tables: as delta -> 0 the 1D tables concentrate on their diagonal
  // (a node only sees the part of the source polynomial within a few sqrt(delta)), so each row
  // keeps only its entries above eta * (largest entry of its source level's tables), eta =
  // 1e-7 eps_pw (a row's dropped part is then below k^3 eta of the pair's magnitude in 3D,
  // k <= 32).  A pair with an all-zero table along some axis contributes nothing and is dropped.
  const size_t ntables = ntab.size() / std::max<size_t>(kk2, 1);
  std::vector<int16_t> nband(ntables * k * 2, 0);
  std::vector<char> tab_empty(ntables, 0);
  {
    std::vector<double> level_max;
    for (size_t t = 0; t < n_std_tables; ++t) {
      if ((size_t)tab_ls[t] >= level_max.size()) level_max.resize(tab_ls[t] + 1, 0.0);
      for (size_t e = 0; e < kk2; ++e) level_max[tab_ls[t]] = std::max(level_max[tab_ls[t]], std::fabs(ntab[t * kk2 + e]));
    }
    for (size_t t = 0; t < ntables; ++t) {
      const double mx = (size_t)tab_ls[t] < level_max.size() ? level_max[tab_ls[t]] : 0.0;
      const double thr = 1e-7 * P.eps_pw * mx;
      bool any = false;
      for (int r = 0; r < k; ++r) {
        int lo = k, hi = -1;
        for (int jj = 0; jj < k; ++jj)
          if (std::fabs(ntab[t * kk2 + (size_t)r * k + jj]) > thr) { lo = std::min(lo, jj); hi = jj; }
        nband[(t * k + r) * 2] = (int16_t)lo;
        nband[(t * k + r) * 2 + 1] = (int16_t)hi;
        any = any || hi >= lo;
      }
      tab_empty[t] = any ? 0 : 1;
    }
  }
  std::vector<fgt::NearPair> npairs;
  npairs.reserve(raw.size());
  for (const fgt::NearPair &pr : raw) {
    bool empty = false;
    for (int a = 0; a < d; ++a) empty = empty || tab_empty[(size_t)pr.tab[a]];
    if (!empty) npairs.push_back(pr);
  }
  ex.n_near_pairs = (int64_t)npairs.size();
  P.n_near_pairs = ex.n_near_pairs;
  {
    bool acc_blocks = false;
    for (const fgt::Block &b : eblocks) acc_blocks = acc_blocks || (b.flags & 1);
    ex.zero_u = (ex.n_near_pairs > 0 || acc_blocks) ? 1 : 0;
  }
  ex.n_points = P.n_targets() * (int64_t)P.np();
  // packed FP32 sigma for the tensor-core form (every block_leaves entry, tagged with its block)
  std::vector<int32_t> pblock;
  bool use_sigp = false;
  for (const fgt::LaunchRange &lr : ex.f2_ranges) use_sigp = use_sigp || lr.tensor;
  if (use_sigp) {
    pblock.resize(bleaves.size());
    for (size_t b = 0; b < blocks.size(); ++b) {
      const int64_t nb = (int64_t)1 << (d * blocks[b].dl);
      for (int64_t j = 0; j < nb; ++j) pblock[(size_t)(blocks[b].leaf0 + j)] = (int32_t)b;
    }
  }
  ex.n_pack = (int64_t)pblock.size();

  // ---- upload
  const size_t o_blocks = pack.add("blocks", blocks), o_bleaves = pack.add("block_leaves", bleaves);
  const size_t o_ebleaves = pack.add("eval_block_leaves", ebleaves);
  const size_t o_pblock = pack.add("pack_block", pblock);
  const size_t o_f1 = pack.add("form1_blocks", f1), o_f2 = pack.add("form2_blocks", f2),
               o_f2p = pack.add("form2_groups", f2ptr), o_e1 = pack.add("eval1_blocks", e1),
               o_e2 = pack.add("eval2_blocks", e2);
  const size_t o_Ff = pack.add("Ff", Ff), o_Fh = pack.add("Fh", Fh), o_Ef = pack.add("Ef", Ef),
               o_Eh = pack.add("Eh", Eh);
  const size_t o_gdst = pack.add("gather_dst", gdst), o_gptr = pack.add("gather_ptr", gptr),
               o_gsrc = pack.add("gather_src", gsrc);
  const size_t o_Pf = pack.add("Pf", Pf), o_Ph = pack.add("Ph", Ph);
  const size_t o_gseg = pack.add("gather_segs", gsegs);
  const size_t o_ntgt = pack.add("near_tgt", ntgt), o_nflags = pack.add("near_flags", nflags),
               o_nptr = pack.add("near_ptr", nptr), o_nsrc = pack.add("near_src", nsrc),
               o_ntab = pack.add("near_tab", ntab), o_npairs = pack.add("near_pairs", npairs);
  const size_t o_nband = pack.add("near_band", nband);
  size_t o_ozj[6], o_ozs[6];
  for (int kind = 0; kind < 6; ++kind) {
    o_ozj[kind] = pack.add("oz_jobs" + std::to_string(kind), ozjobs[kind]);
    o_ozs[kind] = pack.add("oz_slice_jobs" + std::to_string(kind), ozsjobs[kind]);
  }
  const size_t o_oztab = pack.add("oz_btab", oztab), o_ozexp = pack.add("oz_bexp", ozexp);
  const size_t o_eblocks = pack.add("eval_blocks", eblocks);
  const size_t o_ozg = pack.add("oz_groups", ozgroups);
  const size_t o_ggrid = pack.add("gather_grid", ggrid);
  std::vector<std::tuple<size_t, size_t, size_t, int64_t>> step_off;  // items, qf, qh, n
  for (size_t i = 0; i < merge_h.size(); ++i) {
    auto &s = merge_h[i];
    const std::string b = "merge" + std::to_string(i) + "_";
    step_off.emplace_back(pack.add(b + "items", s.items), pack.add(b + "qf", s.qf), pack.add(b + "qh", s.qh),
                          (int64_t)s.items.size());
  }
  for (size_t i = 0; i < push_h.size(); ++i) {
    auto &s = push_h[i];
    const std::string b = "push" + std::to_string(i) + "_";
    step_off.emplace_back(pack.add(b + "items", s.items), pack.add(b + "qf", s.qf), pack.add(b + "qh", s.qh),
                          (int64_t)s.items.size());
  }

  const size_t slot_bytes = sizeof(C) * (size_t)ex.slot_size;
  const size_t psi_slot_bytes =
      ex.psi_pitch > 0 ? sizeof(C) * (size_t)nh * ex.psi_pitch * ex.psi_pitch : slot_bytes;
  const size_t phi_bytes = slot_bytes * (size_t)ex.n_phi_slots, psi_bytes = psi_slot_bytes * (size_t)ex.n_psi_slots;
  const size_t psi_off = (phi_bytes + 255) & ~(size_t)255, sigp_off = (psi_off + psi_bytes + 255) & ~(size_t)255;
  const size_t sigp_bytes = sizeof(float) * (size_t)ex.n_pack * P.np();
  // tcgen05 evaluation: the expansions it reads, once more in the tensor cores' operand layout
  bool use_tc6 = false;
  for (const fgt::LaunchRange &lr : ex.e2_ranges) use_tc6 = use_tc6 || lr.tensor == 4;
  const int64_t tc6_slots = P.fourier ? ex.n_phi_slots : ex.n_psi_slots;
  const size_t ptc_off = (sigp_off + sigp_bytes + 255) & ~(size_t)255;
  const size_t ptc_bytes = use_tc6 ? fgt::eval6_slot_bytes(n1, nh) * (size_t)tc6_slots : 0;
  ex.n_psi_tc_slots = use_tc6 ? tc6_slots : 0;
  // sliced FP64 stages: their two intermediate arrays
  const size_t oz_off = (ptc_off + ptc_bytes + 255) & ~(size_t)255;
  const size_t oz_x_bytes = 2 * sizeof(double) * (size_t)oz_scr;
  const size_t oz_dig_off = (oz_off + oz_x_bytes + 1023) & ~(size_t)1023;
  const size_t oz_rexp_off = (oz_dig_off + (size_t)oz_dig + 255) & ~(size_t)255;
  const size_t oz_bytes = oz_scr > 0 ? oz_rexp_off + sizeof(int) * (size_t)oz_rexp - oz_off : 0;
  fill_flops(P, ex, blocks, merge_h.size() + push_h.size() ? [&] {
    int64_t sf = 0;
    for (auto &s : merge_h) sf += 8 * (int64_t)s.items.size() * nc * ex.slot_size;
    for (auto &s : push_h) sf += 8 * (int64_t)s.items.size() * nc * ex.slot_size;
    return sf;
  }() : 0, anchors.size());
  P.info.device_bytes = (int64_t)(pack.size + oz_off + oz_bytes);
  P.info.n_merge_items = P.info.n_push_items = 0;
  for (auto &s : merge_h) P.info.n_merge_items += (int64_t)s.items.size();
  for (auto &s : push_h) P.info.n_push_items += (int64_t)s.items.size();
  if (!upload) {
    P.ex = ex;
    P.host_pack = std::move(pack);
    P.dirty = false;
    return FGT_OK;
  }
  if (P.dev) { cudaFree(P.dev); P.dev = nullptr; P.dev_bytes = 0; }
  if (P.work) { cudaFree(P.work); P.work = nullptr; P.work_bytes = 0; }
  cudaError_t e = cudaMalloc(&P.dev, std::max<size_t>(pack.size, 256));
  if (e != cudaSuccess) { P.dev = nullptr; return e == cudaErrorMemoryAllocation ? fail(FGT_ERR_OOM, "device tables") : cuda_fail(e, "cudaMalloc"); }
  P.dev_bytes = pack.size;
  for (auto &pt : pack.parts)
    if (!pt.second.empty()) {
      e = cudaMemcpy((char *)P.dev + pt.first, pt.second.data(), pt.second.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "upload");
    }
  P.work_bytes = oz_off + oz_bytes;
  if (P.work_bytes) {
    e = cudaMalloc(&P.work, P.work_bytes);
    if (e != cudaSuccess) {
      P.work = nullptr;
      const size_t want = P.work_bytes;
      P.work_bytes = 0;
      cudaGetLastError();
      return fail(FGT_ERR_OOM, "expansion workspace of " + std::to_string(want) + " bytes");
    }
  }
  auto at = [&](size_t off) { return (const void *)((const char *)P.dev + off); };
  ex.phi = P.work;
  ex.psi = (char *)P.work + psi_off;
  ex.psi_map_ready = 0;
  if (ex.psi_pitch > 0) {
    // the padding of the tcgen05 evaluation's layout is never written: zero it once
    e = cudaMemset(ex.psi, 0, psi_bytes);
    if (e == cudaSuccess) e = fgt::encode_psi_map(ex);
    if (e != cudaSuccess) return cuda_fail(e, "tensor map of the expansions");
    ex.psi_map_ready = 1;
  }
  ex.sigp = sigp_bytes ? (float *)((char *)P.work + sigp_off) : nullptr;
  ex.psi_tc = ptc_bytes ? (void *)((char *)P.work + ptc_off) : nullptr;
  ex.oz_x = oz_bytes ? (double *)((char *)P.work + oz_off) : nullptr;
  ex.oz_y = oz_bytes ? ex.oz_x + oz_scr : nullptr;
  ex.oz_dig = oz_bytes ? (unsigned char *)P.work + oz_dig_off : nullptr;
  ex.oz_rexp = oz_bytes ? (int *)((char *)P.work + oz_rexp_off) : nullptr;
  for (int kind = 0; kind < 6; ++kind) {
    ex.oz_jobs[kind] = (const fgt::OzJob *)at(o_ozj[kind]);
    ex.oz_sjobs[kind] = (const fgt::OzJob *)at(o_ozs[kind]);
  }
  ex.oz_btab = (const unsigned char *)at(o_oztab);
  ex.oz_bexp = (const int32_t *)at(o_ozexp);
  ex.eval_blocks = (const fgt::Block *)at(o_eblocks);
  ex.oz_groups = (const fgt::OzGroup *)at(o_ozg);
  ex.gather_grid = ex.grid_nb > 0 ? (const int32_t *)at(o_ggrid) : nullptr;
  ex.sig_maps_ready = 0;
  if (ex.sig_order == 1) {
    // the tensor maps over the packed density (its address is set just above)
    if (!ex.sigp) return fail(FGT_ERR_STATE, "tcgen05 form without a packed density");
    bool used[3] = {false, false, false};
    for (const fgt::LaunchRange &lr : ex.f2_ranges)
      if (lr.tensor == 7) used[lr.K == 8 ? 0 : lr.K == 16 ? 1 : 2] = true;
    e = fgt::encode_sig_maps(ex, ex.n_pack * (int64_t)P.np(), used);
    if (e != cudaSuccess) return cuda_fail(e, "tensor maps of the packed density");
    ex.sig_maps_ready = 1;
  }
  ex.pack_block = (const int32_t *)at(o_pblock);
  ex.blocks = (const fgt::Block *)at(o_blocks);
  ex.f1_blocks = (const fgt::Block *)at(o_f1);
  ex.f2_blocks = (const fgt::Block *)at(o_f2);
  ex.f2_gptr = (const int32_t *)at(o_f2p);
  ex.e1_blocks = (const fgt::Block *)at(o_e1);
  ex.e2_blocks = (const fgt::Block *)at(o_e2);
  ex.block_leaves = (const int64_t *)at(o_bleaves);
  ex.eval_leaves = (const int64_t *)at(o_ebleaves);
  ex.Ff = at(o_Ff); ex.Fh = at(o_Fh); ex.Ef = at(o_Ef); ex.Eh = at(o_Eh);
  ex.gather_dst = (const int32_t *)at(o_gdst);
  ex.gather_segs = (const fgt::GatherSeg *)at(o_gseg);
  ex.gather_ptr = (const int64_t *)at(o_gptr);
  ex.gather_src = (const fgt::GatherSrc *)at(o_gsrc);
  ex.Pf = at(o_Pf); ex.Ph = at(o_Ph);
  ex.near_tgt = (const int64_t *)at(o_ntgt);
  ex.near_flags = (const int32_t *)at(o_nflags);
  ex.near_ptr = (const int64_t *)at(o_nptr);
  ex.near_src = (const fgt::NearSrc *)at(o_nsrc);
  ex.near_tab = (const double *)at(o_ntab);
  ex.near_pairs = (const fgt::NearPair *)at(o_npairs);
  ex.near_band = (const int16_t *)at(o_nband);
  size_t si = 0;
  for (size_t s = 0; s < merge_h.size(); ++s, ++si) {
    fgt::ShiftStep st;
    st.items = (const fgt::TreeShift *)at(std::get<0>(step_off[si]));
    st.qf = at(std::get<1>(step_off[si]));
    st.qh = at(std::get<2>(step_off[si]));
    st.n = std::get<3>(step_off[si]);
    ex.merge.push_back(st);
  }
  for (size_t s = 0; s < push_h.size(); ++s, ++si) {
    fgt::ShiftStep st;
    st.items = (const fgt::TreeShift *)at(std::get<0>(step_off[si]));
    st.qf = at(std::get<1>(step_off[si]));
    st.qh = at(std::get<2>(step_off[si]));
    st.n = std::get<3>(step_off[si]);
    ex.push.push_back(st);
  }
  const bool multi_form = (ex.n_f1 > 0) + ex.f2_ranges.size() > 1;
  const bool multi_eval = (ex.n_e1 > 0) + ex.e2_ranges.size() > 1;
  if (ex.n_near_pairs > 0 || multi_form || multi_eval) {  // side streams, made once per plan
    for (int i = 0; i < fgt::kSides && !P.side[i]; ++i) {
      e = cudaStreamCreateWithFlags(&P.side[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.fork_ev[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.join_ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "side streams");
    }
    for (int i = 0; i < fgt::kSides; ++i) {
      ex.side[i] = P.side[i];
      ex.fork_ev[i] = P.fork_ev[i];
      ex.join_ev[i] = P.join_ev[i];
    }
    // default: forked before the gather, so that the near field's FP64 work overlaps the L2-bound
    // gather and the evaluation rather than the form (fastest of the three fork points measured)
    ex.near_phase = (P.tune.near_phase == 0 || P.tune.near_phase == 4) ? P.tune.near_phase : 2;
  }
  P.ex = ex;

  P.dirty = false;
  return FGT_OK;
}

fgt_status prepare(fgt_plan &P, bool upload = true) {
  if (P.prec == FGT_PREC_SPLIT) return prepare_typed<float2>(P, upload);
  return prepare_typed<double2>(P, upload);
}

fgt_status create_impl(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                       const fgt_tree *tree, fgt_plan **out, bool upload = true) {
  if (!out) return fail(FGT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (d != 2 && d != 3) return fail(FGT_ERR_ARG, "d must be 2 or 3");
  if (!tree || tree->d != d) return fail(FGT_ERR_ARG, "tree missing or tree->d != d");
  if (tree->k < 1 || tree->k > fgt::kMaxK) return fail(FGT_ERR_ARG, "k must be in [1, 16]");
  if (tree->n_leaves < 1 || !tree->leaf_level || !tree->leaf_coord) return fail(FGT_ERR_ARG, "empty tree");
  if (!(delta > 0) || !std::isfinite(delta)) return fail(FGT_ERR_ARG, "delta must be positive");
  if (!(tol >= 1e-14 && tol <= 1e-1)) return fail(FGT_ERR_ARG, "tol must be in [1e-14, 1e-1]");
  if (bc != FGT_BC_FREE && bc != FGT_BC_PERIODIC) return fail(FGT_ERR_ARG, "bad bc");
  if (prec != FGT_PREC_FP64 && prec != FGT_PREC_SPLIT && prec != FGT_PREC_FP64_TC)
    return fail(FGT_ERR_ARG, "bad precision");
  if (prec == FGT_PREC_SPLIT && tol < 1e-7) return fail(FGT_ERR_ARG, "split precision needs tol >= 1e-7");
  if (mode != FGT_MODE_FUSED && mode != FGT_MODE_HIERARCHICAL) return fail(FGT_ERR_ARG, "bad mode");
  fgt_plan *P = new (std::nothrow) fgt_plan();
  if (!P) return fail(FGT_ERR_OOM, "host allocation");
  P->d = d; P->k = tree->k; P->bc = bc; P->prec = prec; P->mode = mode;
  P->delta = delta; P->tol = tol; P->eps_pw = eps_pw > 0 ? eps_pw : tol;
  {
    const char *tc = std::getenv("FGT_TC_EVAL");
    P->tc_eval = tc && tc[0] == '1';
    const char *tc4 = std::getenv("FGT_TC_EVAL4");
    P->tc_eval4 = tc4 && tc4[0] == '1';
    // the evaluation with the half-range axis last: default in FP64 (fewer FP64 products, 10-35 %
    // faster there), in split precision only with FGT_EVAL5=1 (measured no faster: issue-bound)
    const char *e5 = std::getenv("FGT_EVAL5");
    P->eval5 = e5 ? e5[0] == '1' : prec == FGT_PREC_FP64;
    // evaluation stage 1 on tcgen05 (split precision, K <= 16): opt-in with FGT_TC_EVAL6=1; measured
    // slower than the CUDA-core kernel on GB300 (stages 2-3 dominate, and every CTA streams the
    // split expansion, twice the bytes of the FP32 one, from L2)
    const char *t6 = std::getenv("FGT_TC_EVAL6");
    P->tc_eval6 = t6 && t6[0] == '1';
    // all three evaluation contractions on tcgen05 with tensor-map staged expansions (split
    // precision, 3D, blocks of K = 8, 16, 32, n1 <= 32): the default where it applies (measured
    // 1.7x faster than the CUDA-core evaluation on the 16.8M-point periodic workload);
    // FGT_EVAL7=0 turns it off
    const char *e7 = std::getenv("FGT_EVAL7");
    P->eval7 = !(e7 && e7[0] == '0');
    // all three form contractions on tcgen05 (split precision, 3D, n1 <= 32): by default for blocks of
    // K = 16 and 32 (measured 1.4x faster than the CUDA-core form on the 16.8M-point periodic
    // workload; for K = 8 blocks slower), FGT_FORM7=1 for K = 8 as well, FGT_FORM7=0 for none
    const char *f7 = std::getenv("FGT_FORM7");
    P->form7 = !(f7 && f7[0] == '0');
    P->form7_k8 = f7 && f7[0] == '1';
    // FP64-accurate form and evaluation on the BF16 tensor cores by exact slicing (precision
    // FP64_TC, 3D, fused mode, n1 <= 80): the default there; FGT_OZAKI=0 keeps the DMMA kernels
    const char *oz = std::getenv("FGT_OZAKI");
    P->ozaki = !(oz && oz[0] == '0');
    // the run-form gather for the FP64 expansions too (measured 2.0x faster than the per-anchor
    // gather on the 16.8M-point periodic workload at tol 1e-10, 1.7x on the 2.09M-point adaptive
    // one); FGT_GATHER2=0 keeps the per-anchor kernel
    const char *g2 = std::getenv("FGT_GATHER2");
    P->gather2_fp64 = !(g2 && g2[0] == '0');
    const char *g3 = std::getenv("FGT_GATHER3");
    P->gather3 = !(g3 && g3[0] == '0');
  }
  P->n_leaves = tree->n_leaves;
  P->leaf_level.assign(tree->leaf_level, tree->leaf_level + tree->n_leaves);
  P->leaf_coord.assign(tree->leaf_coord, tree->leaf_coord + tree->n_leaves * d);
  fgt_status s = build_tree(*P);
  if (s != FGT_OK) { delete P; return s; }
  // parameters
  choose_params(delta, P->eps_pw, bc, P->lc, P->D0, P->R, P->h, P->M, P->n_p, P->fourier);
  P->n_f = 2 * P->M;
  if (P->fourier) {
    P->M = P->n_p + 1;     // modes -n_p..n_p
    P->kappa = 2.0 * kPi;
    P->n_f = 0;
  } else {
    P->kappa = P->h / std::sqrt(delta);
    P->n_p = 0;
  }
  P->n1 = 2 * P->M - 1;
  P->nh = P->M;
  P->wmode.resize(P->n1);
  for (int a = 0; a < P->n1; ++a) {
    const int m = a - (P->M - 1);
    P->wmode[a] = P->fourier ? std::sqrt(kPi * delta) * std::exp(-kPi * kPi * delta * m * m)
                             : P->h / (2.0 * std::sqrt(kPi)) * std::exp(-0.25 * m * m * P->h * P->h);
  }
  // f flags (Definition fflagdef); Fourier mode: every leaf is evaluated from the root series
  for (Box &b : P->boxes) b.f = 0;
  if (P->fourier) {
    for (Box &b : P->boxes) b.f = 1;
  } else {
    const int nb = 1 << P->lc;
    int noff = 1;
    for (int a = 0; a < d; ++a) noff *= 3;
    for (Box &b : P->boxes) {
      if (b.level > P->lc) { b.f = 1; continue; }
      if (b.level < P->lc) continue;
      for (int oc = 0; oc < noff && !b.f; ++oc) {
        int32_t q[3] = {0, 0, 0};
        bool ok = true;
        for (int a = 0, r = oc; a < d; ++a, r /= 3) {
          int v = b.c[a] + r % 3 - 1;
          if (v < 0 || v >= nb) {
            if (bc != FGT_BC_PERIODIC) { ok = false; break; }
            v = (v + nb) % nb;
          }
          q[a] = v;
        }
        if (!ok) continue;
        const int32_t S = P->find(P->lc, q);
        if (S >= 0 && P->boxes[S].leaf < 0) b.f = 1;
      }
    }
  }
  // quadrature and values -> coefficients
  P->eta.resize(P->k);
  P->weta.resize(P->k);
  fgt::gl_rule(P->k, P->eta.data(), P->weta.data());
  P->Tvp.resize((size_t)P->k * P->k);
  fgt::val_to_pol(P->k, P->eta.data(), P->weta.data(), P->Tvp.data());
  s = prepare(*P, upload);
  if (s != FGT_OK) { delete P; return s; }
  *out = P;
  return FGT_OK;
}

void fill_info(const fgt_plan &P, fgt_plan_info &I) {
  I.d = P.d; I.k = P.k; I.bc = P.bc;
  I.cutoff_level = P.lc; I.fourier = P.fourier; I.max_level = P.lmax;
  I.n_f = P.n_f; I.n_p = P.n_p; I.modes_1d = P.n1; I.modes_half = P.nh;
  I.delta = P.delta; I.tol = P.tol; I.eps_pw = P.eps_pw;
  I.D0 = P.D0; I.R = P.R; I.h = P.h;
  I.n_leaves = P.n_leaves; I.n_boxes = (int64_t)P.boxes.size();
  int64_t npw = 0;
  for (int64_t i = 0; i < P.n_leaves; ++i) npw += P.boxes[P.leaf_box[i]].f ? 1 : 0;
  I.n_pw_leaves = npw;
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

fgt_status fgt_plan_create_ex(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                              const fgt_tree *tree, fgt_plan **out) {
  try {
    return create_impl(d, delta, tol, eps_pw, bc, prec, mode, tree, out);
  } catch (const std::bad_alloc &) {
    return fail(FGT_ERR_OOM, "host allocation");
  } catch (...) {
    return fail(FGT_ERR_ARG, "unexpected host exception");
  }
}

fgt_status fgt_plan_analyze(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                            const fgt_tree *tree, fgt_plan_info *info) {
  if (!info) return fail(FGT_ERR_ARG, "info is NULL");
  try {
    fgt_plan *P = nullptr;
    fgt_status s = create_impl(d, delta, tol, eps_pw, bc, prec, mode, tree, &P, false);
    if (s != FGT_OK) return s;
    *info = P->info;
    fill_info(*P, *info);
    delete P;
    return FGT_OK;
  } catch (const std::bad_alloc &) {
    return fail(FGT_ERR_OOM, "host allocation");
  }
}

fgt_status fgt_plan_create_host(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                                const fgt_tree *tree, fgt_plan **out) {
  try {
    fgt_status s = create_impl(d, delta, tol, eps_pw, bc, prec, mode, tree, out, false);
    if (s == FGT_OK) (*out)->host_only = true;
    return s;
  } catch (const std::bad_alloc &) {
    return fail(FGT_ERR_OOM, "host allocation");
  }
}

fgt_status fgt_plan_host_array(const fgt_plan *plan, const char *name, const void **data, size_t *bytes) {
  if (!plan || !name || !data || !bytes) return fail(FGT_ERR_ARG, "NULL argument");
  if (!plan->host_only) return fail(FGT_ERR_STATE, "host arrays are kept only by host-only plans");
  const DevPack &pk = plan->host_pack;
  for (size_t i = 0; i < pk.names.size(); ++i)
    if (pk.names[i] == name) {
      *data = pk.parts[i].second.data();
      *bytes = pk.parts[i].second.size();
      return FGT_OK;
    }
  return fail(FGT_ERR_ARG, std::string("no host array named ") + name);
}

fgt_status fgt_plan_create(int d, double delta, double tol, int bc, const fgt_tree *tree, fgt_plan **out) {
  return fgt_plan_create_ex(d, delta, tol, 0.0, bc, FGT_PREC_FP64, FGT_MODE_FUSED, tree, out);
}

fgt_status fgt_plan_set_precision(fgt_plan *plan, int prec) {
  if (!plan) return fail(FGT_ERR_ARG, "plan is NULL");
  if (prec != FGT_PREC_FP64 && prec != FGT_PREC_SPLIT && prec != FGT_PREC_FP64_TC)
    return fail(FGT_ERR_ARG, "bad precision");
  if (prec == FGT_PREC_SPLIT && plan->tol < 1e-7) return fail(FGT_ERR_ARG, "split precision needs tol >= 1e-7");
  if (plan->prec != prec) { plan->prec = prec; plan->dirty = true; }
  return FGT_OK;
}

fgt_status fgt_plan_set_mode(fgt_plan *plan, int mode) {
  if (!plan) return fail(FGT_ERR_ARG, "plan is NULL");
  if (mode != FGT_MODE_FUSED && mode != FGT_MODE_HIERARCHICAL) return fail(FGT_ERR_ARG, "bad mode");
  if (plan->mode != mode) { plan->mode = mode; plan->dirty = true; }
  return FGT_OK;
}

fgt_status fgt_plan_get_info(const fgt_plan *plan, fgt_plan_info *info) {
  if (!plan || !info) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->dirty) {
    try {
      fgt_status s = prepare(*const_cast<fgt_plan *>(plan), !plan->host_only);
      if (s != FGT_OK) return s;
    } catch (...) {
      return fail(FGT_ERR_OOM, "host allocation");
    }
  }
  *info = plan->info;
  fill_info(*plan, *info);
  return FGT_OK;
}

size_t fgt_plan_device_bytes(const fgt_plan *plan) {
  if (!plan) return 0;
  return plan->dev_bytes + plan->work_bytes + (plan->stage ? sizeof(double) * plan->stage_elems : 0);
}

fgt_status fgt_execute_async(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream) {
  if (!plan || !sigma_dev || !u_dev) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->host_only) return fail(FGT_ERR_STATE, "host-only plan cannot execute");
  if (plan->dirty) {
    fgt_status s;
    try {
      s = prepare(*plan);
    } catch (...) {
      return fail(FGT_ERR_OOM, "host allocation");
    }
    if (s != FGT_OK) return s;
  }
  plan->ex.events = nullptr;
  if (plan->profiling) {
    const size_t need = plan->ev_used + 2 * fgt::kPhases;
    while (plan->ev_pool.size() < need) {
      cudaEvent_t ev;
      cudaError_t ce = cudaEventCreate(&ev);
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaEventCreate");
      plan->ev_pool.push_back(ev);
    }
    plan->ex.events = plan->ev_pool.data() + plan->ev_used;
    plan->ev_used = need;
  }
  {  // checked build: the buffers this transform may touch (a no-op otherwise)
    const size_t np = (size_t)plan->np();
    const void *b[4] = {sigma_dev, u_dev, plan->dev, plan->work};
    const size_t n[4] = {8 * np * (size_t)plan->n_leaves, 8 * np * (size_t)plan->n_targets(), plan->dev_bytes,
                         plan->work_bytes};
    cudaError_t ce = fgt::set_check_ranges(b, n, 4, (cudaStream_t)stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "check ranges");
  }
  cudaError_t e = fgt::run_transform(plan->ex, sigma_dev, u_dev, (cudaStream_t)stream);
  plan->ex.events = nullptr;
  if (e != cudaSuccess) return cuda_fail(e, "transform launch");
  return FGT_OK;
}

fgt_status fgt_plan_set_output_tree(fgt_plan *plan, const fgt_tree *out) {
  if (!plan) return fail(FGT_ERR_ARG, "plan is NULL");
  if (!out || out->n_leaves == 0) {
    if (plan->n_out) plan->dirty = true;
    plan->n_out = 0;
    plan->out_level.clear(); plan->out_coord.clear(); plan->out_src.clear();
    return FGT_OK;
  }
  const int d = plan->d;
  if (out->d != d || out->k != plan->k || out->n_leaves < 0 || !out->leaf_level || !out->leaf_coord)
    return fail(FGT_ERR_ARG, "output tree: dimension, k or arrays do not match the plan");
  if (plan->lmax > 20) return fail(FGT_ERR_ARG, "output trees need source leaves at levels <= 20");
  if (plan->mode == FGT_MODE_HIERARCHICAL) return fail(FGT_ERR_ARG, "output trees need the fused mode");
  const int64_t n = out->n_leaves;
  std::vector<int64_t> src(n);
  std::unordered_map<uint64_t, int64_t> seen;
  for (int64_t i = 0; i < n; ++i) {
    const int lt = out->leaf_level[i];
    if (lt < 0 || lt > 20) return fail(FGT_ERR_TREE, "output tree: level out of range [0, 20]");
    int32_t c[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      c[a] = out->leaf_coord[i * d + a];
      if (c[a] < 0 || c[a] >= (1 << lt)) return fail(FGT_ERR_TREE, "output tree: coordinate out of range");
    }
    if (!seen.emplace(box_key(lt, c), i).second) return fail(FGT_ERR_TREE, "output tree: repeated leaf");
    int64_t leaf = -1;
    for (int l = lt; l >= 0 && leaf < 0; --l) {
      int32_t q[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) q[a] = c[a] >> (lt - l);
      const int32_t b = plan->find(l, q);
      if (b >= 0) {
        if (plan->boxes[b].leaf < 0) break;  // lies above a source leaf: coarser than the source tree
        leaf = plan->boxes[b].leaf;
      }
    }
    if (leaf < 0) return fail(FGT_ERR_TREE, "output tree: a leaf is not inside one source leaf");
    src[i] = leaf;
  }
  for (int64_t i = 0; i < n; ++i) {  // no output leaf inside another
    for (int l = out->leaf_level[i] - 1; l >= plan->leaf_level[src[i]]; --l) {
      int32_t q[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) q[a] = out->leaf_coord[i * d + a] >> (out->leaf_level[i] - l);
      if (seen.count(box_key(l, q))) return fail(FGT_ERR_TREE, "output tree: overlapping leaves");
    }
  }
  // the output leaves need not cover the source leaves: u is evaluated at the given leaves only
  // (Algorithm 5 re-evaluates the subdivided leaves alone)
  plan->n_out = n;
  plan->out_level.assign(out->leaf_level, out->leaf_level + n);
  plan->out_coord.assign(out->leaf_coord, out->leaf_coord + n * d);
  plan->out_src = std::move(src);
  plan->dirty = true;
  return FGT_OK;
}

// ---------------------------------------------------------------------------- Algorithm 3 on the GPU

struct fgt_built_tree {
  int d = 0, k = 0;
  std::vector<int32_t> level, coord;
  double *sigma = nullptr;  // device [n][k^d]
  ~fgt_built_tree() {
    if (sigma) cudaFree(sigma);
  }
};

namespace {

// 2:1 balance (boxes sharing a boundary point, corners included, across the wrap when periodic):
// a leaf with a neighbour leaf two or more levels coarser splits that neighbour, until none does.
void balance_tree(int d, bool periodic, std::vector<int32_t> &level, std::vector<int32_t> &coord) {
  struct Key { int l; int32_t c[3]; };
  std::unordered_map<uint64_t, Key> leaves;
  std::vector<Key> queue;
  for (size_t i = 0; i < level.size(); ++i) {
    Key kk{level[i], {0, 0, 0}};
    for (int a = 0; a < d; ++a) kk.c[a] = coord[i * d + a];
    leaves.emplace(box_key(kk.l, kk.c), kk);
    queue.push_back(kk);
  }
  int noff = 1;
  for (int a = 0; a < d; ++a) noff *= 3;
  while (!queue.empty()) {
    const Key t = queue.back();
    queue.pop_back();
    if (!leaves.count(box_key(t.l, t.c))) continue;
    const int n = 1 << t.l;
    for (int oc = 0; oc < noff; ++oc) {
      int32_t q[3] = {0, 0, 0};
      bool ok = true, self = true;
      for (int a = 0, r = oc; a < d; ++a, r /= 3) {
        const int o = r % 3 - 1;
        self = self && o == 0;
        int v = t.c[a] + o;
        if (v < 0 || v >= n) {
          if (!periodic) { ok = false; break; }
          v = (v % n + n) % n;
        }
        q[a] = v;
      }
      if (!ok || self) continue;
      // the leaf covering the neighbour position at level t.l, if it is coarser
      for (int up = 2; up <= t.l; ++up) {
        int32_t pc[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) pc[a] = q[a] >> up;
        auto it = leaves.find(box_key(t.l - up, pc));
        if (it == leaves.end()) continue;
        const Key s = it->second;
        leaves.erase(it);
        for (int ch = 0; ch < (1 << d); ++ch) {
          Key kid{s.l + 1, {0, 0, 0}};
          for (int a = 0; a < d; ++a) kid.c[a] = 2 * s.c[a] + ((ch >> a) & 1);
          leaves.emplace(box_key(kid.l, kid.c), kid);
          queue.push_back(kid);
        }
        queue.push_back(t);
        break;
      }
    }
  }
  std::vector<std::pair<uint64_t, Key>> all(leaves.begin(), leaves.end());
  std::sort(all.begin(), all.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
  level.clear();
  coord.clear();
  for (const auto &e : all) {
    level.push_back(e.second.l);
    for (int a = 0; a < d; ++a) coord.push_back(e.second.c[a]);
  }
}

}  // namespace

fgt_status fgt_build_gaussian_tree(int d, int k, int n_gauss, const double *centers, const double *alphas,
                                   const double *amps, int periodic, double eps, int min_level, int max_level,
                                   void *stream, fgt_built_tree **out) {
  if (!out) return fail(FGT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if ((d != 2 && d != 3) || k < 1 || k > fgt::kMaxLeafK || n_gauss < 1 || !centers || !alphas || !(eps > 0) ||
      min_level < 0 || max_level < min_level || max_level > 20)
    return fail(FGT_ERR_ARG, "build tree: bad arguments (d 2/3, 1 <= k <= 16, 0 <= min <= max <= 20)");
  for (int i = 0; i < n_gauss; ++i)
    if (!(alphas[i] > 0)) return fail(FGT_ERR_ARG, "build tree: alphas must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  const int np = d == 3 ? k * k * k : k * k;
  std::vector<double> gp((size_t)n_gauss * (d + 2));
  for (int i = 0; i < n_gauss; ++i) {
    for (int a = 0; a < d; ++a) gp[(size_t)i * (d + 2) + a] = centers[(size_t)i * d + a];
    gp[(size_t)i * (d + 2) + d] = alphas[i];
    gp[(size_t)i * (d + 2) + d + 1] = amps ? amps[i] : 1.0;
  }
  // device scratch, grown as needed
  double *dg = nullptr, *dv = nullptr, *de = nullptr, *ds = nullptr;
  int32_t *dl = nullptr, *dc = nullptr;
  size_t cap = 0;
  auto release = [&]() {
    cudaFree(dg); cudaFree(dv); cudaFree(de); cudaFree(ds); cudaFree(dl); cudaFree(dc);
  };
  auto reserve = [&](size_t n) -> cudaError_t {
    if (n <= cap) return cudaSuccess;
    cudaFree(dv); cudaFree(de); cudaFree(ds); cudaFree(dl); cudaFree(dc);
    dv = de = ds = nullptr; dl = dc = nullptr;
    cap = std::max(n, 2 * cap);
    cudaError_t e = cudaMalloc(&dv, sizeof(double) * cap * np);
    if (e == cudaSuccess) e = cudaMalloc(&de, sizeof(double) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&ds, sizeof(double) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(int32_t) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&dc, sizeof(int32_t) * cap * d);
    return e;
  };
  cudaError_t ce = cudaMalloc(&dg, sizeof(double) * gp.size());
  if (ce == cudaSuccess) ce = cudaMemcpy(dg, gp.data(), sizeof(double) * gp.size(), cudaMemcpyHostToDevice);
  std::vector<int32_t> al(1, 0), ac((size_t)d, 0), ll, lc;  // active boxes, finished leaves
  double leaf_sq = 0.0;
  std::vector<double> err, sq;
  for (int l = 0; ce == cudaSuccess && !al.empty(); ++l) {
    const size_t na = al.size();
    if ((ce = reserve(na)) != cudaSuccess) break;
    ce = cudaMemcpyAsync(dl, al.data(), sizeof(int32_t) * na, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dc, ac.data(), sizeof(int32_t) * na * d, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = fgt::gauss_nodes(d, k, (int64_t)na, dl, dc, n_gauss, dg, periodic, dv, st);
    if (ce == cudaSuccess) ce = fgt::leaf_errors(d, k, (int64_t)na, dv, de, ds, st);
    err.resize(na);
    sq.resize(na);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(err.data(), de, sizeof(double) * na, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(sq.data(), ds, sizeof(double) * na, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) break;
    // ||sigma||_2 over the current partition of B: finished leaves and this level's boxes
    const double vol = std::pow(0.5 * std::ldexp(1.0, -l), d);
    double norm2 = leaf_sq;
    for (size_t i = 0; i < na; ++i) norm2 += sq[i] * vol;
    const double thr = eps * std::sqrt(norm2);
    std::vector<int32_t> nl, nc;
    for (size_t i = 0; i < na; ++i) {
      const bool split = l < max_level && (l < min_level || err[i] > thr);
      if (split) {
        for (int ch = 0; ch < (1 << d); ++ch) {
          nl.push_back(l + 1);
          for (int a = 0; a < d; ++a) nc.push_back(2 * ac[i * d + a] + ((ch >> a) & 1));
        }
      } else {
        ll.push_back(l);
        for (int a = 0; a < d; ++a) lc.push_back(ac[i * d + a]);
        leaf_sq += sq[i] * vol;
      }
    }
    al.swap(nl);
    ac.swap(nc);
  }
  if (ce != cudaSuccess) {
    release();
    return cuda_fail(ce, "build tree");
  }
  balance_tree(d, periodic != 0, ll, lc);
  auto *T = new (std::nothrow) fgt_built_tree();
  if (!T) { release(); return fail(FGT_ERR_OOM, "host allocation"); }
  T->d = d; T->k = k; T->level = ll; T->coord = lc;
  const size_t n = ll.size();
  ce = reserve(n);
  if (ce == cudaSuccess) ce = cudaMalloc(&T->sigma, sizeof(double) * n * np);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(dl, ll.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(dc, lc.data(), sizeof(int32_t) * n * d, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = fgt::gauss_nodes(d, k, (int64_t)n, dl, dc, n_gauss, dg, periodic, T->sigma, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  release();
  if (ce != cudaSuccess) {
    delete T;
    return cuda_fail(ce, "build tree");
  }
  *out = T;
  return FGT_OK;
}

fgt_status fgt_built_tree_get(const fgt_built_tree *t, int64_t *n_leaves, const int32_t **level,
                              const int32_t **coord, const double **sigma_dev) {
  if (!t) return fail(FGT_ERR_ARG, "tree is NULL");
  if (n_leaves) *n_leaves = (int64_t)t->level.size();
  if (level) *level = t->level.data();
  if (coord) *coord = t->coord.data();
  if (sigma_dev) *sigma_dev = t->sigma;
  return FGT_OK;
}

fgt_status fgt_built_tree_copy_sigma(const fgt_built_tree *t, double *dst_dev, void *stream) {
  if (!t || !dst_dev) return fail(FGT_ERR_ARG, "NULL argument");
  const size_t np = t->d == 3 ? (size_t)t->k * t->k * t->k : (size_t)t->k * t->k;
  cudaError_t e = cudaMemcpyAsync(dst_dev, t->sigma, sizeof(double) * np * t->level.size(), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "copy sigma");
}

void fgt_built_tree_destroy(fgt_built_tree *t) { delete t; }

fgt_status fgt_leaf_errors(int d, int k, int64_t n, const double *vals_dev, double *err_dev, double *sumsq_dev,
                           void *stream) {
  if ((d != 2 && d != 3) || k < 1 || k > fgt::kMaxLeafK || n < 0 || (n > 0 && (!vals_dev || !err_dev)))
    return fail(FGT_ERR_ARG, "leaf errors: d must be 2 or 3, 1 <= k <= 16, device arrays given");
  cudaError_t e = fgt::leaf_errors(d, k, n, vals_dev, err_dev, sumsq_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "leaf errors");
}

fgt_status fgt_merge_children(int d, int k, int64_t n_parents, const int64_t *child_rows_dev, const double *vals_dev,
                              double *parent_dev, void *stream) {
  if ((d != 2 && d != 3) || k < 1 || k > fgt::kMaxLeafK || n_parents < 0 ||
      (n_parents > 0 && (!child_rows_dev || !vals_dev || !parent_dev)))
    return fail(FGT_ERR_ARG, "merge children: d must be 2 or 3, 1 <= k <= 16, device arrays given");
  cudaError_t e = fgt::merge_children(d, k, n_parents, child_rows_dev, vals_dev, parent_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "merge children");
}

fgt_status fgt_plan_get_tuning(const fgt_plan *plan, fgt_tuning *out) {
  if (!plan || !out) return fail(FGT_ERR_ARG, "NULL argument");
  *out = plan->tune;
  return FGT_OK;
}

fgt_status fgt_plan_set_tuning(fgt_plan *plan, const fgt_tuning *t) {
  if (!plan || !t) return fail(FGT_ERR_ARG, "NULL argument");
  if (t->eval_rows16 < 1 || t->eval_rows_large < 1 || t->form_group < 1 || t->form_group > 8 ||
      (t->near_phase != 0 && t->near_phase != 2 && t->near_phase != 4))
    return fail(FGT_ERR_ARG, "tuning value out of range");
  const double ms = plan->tune.ms;
  plan->tune = *t;
  plan->tune.ms = ms;
  plan->dirty = true;
  return FGT_OK;
}

fgt_status fgt_plan_autotune(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream, int reps,
                             fgt_tuning *out) {
  if (!plan || !sigma_dev || !u_dev) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->host_only) return fail(FGT_ERR_STATE, "host-only plan cannot execute");
  if (reps < 1) reps = 3;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(ce, "autotune events");
  }
  const bool prof = plan->profiling;
  plan->profiling = false;
  // one timing: re-plan with the candidate knobs, one warm-up, then reps executions
  auto time_it = [&](double *ms) -> fgt_status {
    plan->dirty = true;
    fgt_status s = fgt_execute_async(plan, sigma_dev, u_dev, stream);
    if (s != FGT_OK) return s;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == FGT_OK; ++r) s = fgt_execute_async(plan, sigma_dev, u_dev, stream);
    cudaEventRecord(e1, st);
    if (s != FGT_OK) return s;
    cudaError_t c = cudaEventSynchronize(e1);
    float v = 0.f;
    if (c == cudaSuccess) c = cudaEventElapsedTime(&v, e0, e1);
    if (c != cudaSuccess) return cuda_fail(c, "autotune timing");
    *ms = v / reps;
    return FGT_OK;
  };
  // coordinate descent, one pass, over the knobs that can matter for this plan
  fgt_tuning best = plan->tune;
  double best_ms = 0.0;
  fgt_status s = time_it(&best_ms);
  const bool split3 = plan->d == 3 && plan->prec == FGT_PREC_SPLIT;
  struct Knob { int fgt_tuning::*field; std::vector<int> values; bool on; };
  const Knob knobs[] = {
      {&fgt_tuning::form_group, {2, 4, 8}, plan->mode == FGT_MODE_FUSED},
      {&fgt_tuning::eval_rows16, {4, 8, 16}, split3},
      {&fgt_tuning::eval_rows_large, {4, 8}, split3},
      {&fgt_tuning::near_phase, {0, 2, 4}, plan->n_near_pairs > 0},
  };
  for (const Knob &kb : knobs) {
    if (s != FGT_OK || !kb.on) continue;
    for (int v : kb.values) {
      if (v == best.*kb.field) continue;
      plan->tune = best;
      plan->tune.*kb.field = v;
      double ms = 0.0;
      s = time_it(&ms);
      if (s != FGT_OK) break;
      if (ms < best_ms) { best_ms = ms; best = plan->tune; }
    }
  }
  plan->tune = best;
  plan->tune.ms = best_ms;
  plan->dirty = true;
  plan->profiling = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != FGT_OK) return s;
  try {
    s = prepare(*plan);  // ready to execute with the chosen knobs
  } catch (...) {
    return fail(FGT_ERR_OOM, "host allocation");
  }
  if (s != FGT_OK) return s;
  if (out) *out = plan->tune;
  return FGT_OK;
}

fgt_status fgt_plan_set_profiling(fgt_plan *plan, int on) {
  if (!plan) return fail(FGT_ERR_ARG, "plan is NULL");
  plan->profiling = on != 0;
  plan->ev_used = 0;
  return FGT_OK;
}

fgt_status fgt_plan_read_profile(fgt_plan *plan, double *ms, int *n_transforms) {
  if (!plan || !ms) return fail(FGT_ERR_ARG, "NULL argument");
  for (int p = 0; p < fgt::kPhases; ++p) ms[p] = 0.0;
  const size_t nt = plan->ev_used / (2 * fgt::kPhases);
  for (size_t t = 0; t < nt; ++t)
    for (int p = 0; p < fgt::kPhases; ++p) {
      float v = 0.f;
      cudaEvent_t *ev = plan->ev_pool.data() + t * 2 * fgt::kPhases;
      cudaError_t ce = cudaEventSynchronize(ev[2 * p + 1]);
      if (ce != cudaSuccess) return cuda_fail(ce, "profile");
      ce = cudaEventElapsedTime(&v, ev[2 * p], ev[2 * p + 1]);
      if (ce != cudaSuccess) return cuda_fail(ce, "profile");
      ms[p] += v;
    }
  if (n_transforms) *n_transforms = (int)nt;
  plan->ev_used = 0;
  return FGT_OK;
}

static_assert(fgt::kNoallocScratchBytes == FGT_NOALLOC_SCRATCH_BYTES,
              "the header's scratch size must match the library's array");

fgt_status fgt_execute_noalloc(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream) {
  if (!plan || !sigma_dev || !u_dev) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->host_only) return fail(FGT_ERR_STATE, "host-only plan cannot execute");
  // re-planning would allocate: the plan must already be prepared for its mode and precision
  if (plan->dirty) return fail(FGT_ERR_STATE, "plan changed since it was prepared; run fgt_plan_get_info first");
  const size_t c = plan->f32() ? 8 : 16;
  const size_t phi = c * (size_t)plan->ex.slot_size * (size_t)plan->ex.n_phi_slots;
  const size_t psi = c * (size_t)plan->ex.slot_size * (size_t)plan->ex.n_psi_slots;
  if (((phi + 255) & ~(size_t)255) + psi > fgt::kNoallocScratchBytes)
    return fail(FGT_ERR_ARG, "expansion workspace of " + std::to_string(phi + psi) +
                                 " bytes exceeds the fixed allocation-free scratch of " +
                                 std::to_string(fgt::kNoallocScratchBytes) + " bytes");
  // The scratch array is per device and is looked up for the current device: every buffer must
  // live on the plan's device, which is made current for the call (and restored afterwards).
  int plan_dev = -1;
  {
    cudaPointerAttributes pa{};
    cudaError_t ce = cudaPointerGetAttributes(&pa, plan->dev);
    if (ce != cudaSuccess || pa.type != cudaMemoryTypeDevice) return cuda_fail(ce, "plan device");
    plan_dev = pa.device;
    const void *bufs[2] = {sigma_dev, u_dev};
    for (const void *b : bufs) {
      cudaPointerAttributes ba{};
      ce = cudaPointerGetAttributes(&ba, b);
      if (ce != cudaSuccess) { cudaGetLastError(); return fail(FGT_ERR_ARG, "sigma or u is not device memory"); }
      if (ba.type != cudaMemoryTypeDevice && ba.type != cudaMemoryTypeManaged)
        return fail(FGT_ERR_ARG, "sigma or u is not device memory");
      if (ba.device != plan_dev)
        return fail(FGT_ERR_ARG, "sigma or u is on device " + std::to_string(ba.device) + ", the plan on device " +
                                     std::to_string(plan_dev));
    }
  }
  int cur_dev = -1;
  if (cudaGetDevice(&cur_dev) != cudaSuccess) return fail(FGT_ERR_CUDA, "cudaGetDevice");
  struct DeviceGuard {
    int prev;
    bool switched;
    ~DeviceGuard() { if (switched) cudaSetDevice(prev); }
  } guard{cur_dev, cur_dev != plan_dev};
  if (guard.switched && cudaSetDevice(plan_dev) != cudaSuccess) {
    guard.switched = false;
    return fail(FGT_ERR_CUDA, "cudaSetDevice");
  }
  fgt::ExecDesc ex = plan->ex;
  ex.events = nullptr;
  {  // checked build: sigma, u, the plan's tables and the fixed scratch array
    void *scratch = nullptr;
    cudaError_t ce = fgt::noalloc_scratch(&scratch);
    if (ce != cudaSuccess) return cuda_fail(ce, "allocation-free scratch");
    const size_t np = (size_t)plan->np();
    const void *b[4] = {sigma_dev, u_dev, plan->dev, scratch};
    const size_t n[4] = {8 * np * (size_t)plan->n_leaves, 8 * np * (size_t)plan->n_targets(), plan->dev_bytes,
                         fgt::kNoallocScratchBytes};
    if ((ce = fgt::set_check_ranges(b, n, 4, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(ce, "check ranges");
  }
  cudaError_t e = fgt::run_transform_noalloc(ex, sigma_dev, u_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "allocation-free transform");
  return FGT_OK;
}

fgt_status fgt_execute(fgt_plan *plan, const double *sigma_dev, double *u_dev) {
  fgt_status s = fgt_execute_async(plan, sigma_dev, u_dev, nullptr);
  if (s != FGT_OK) return s;
  cudaError_t e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "transform");
  return FGT_OK;
}

fgt_status fgt_execute_host(fgt_plan *plan, const double *sigma_host, double *u_host, void *stream) {
  if (!plan || !sigma_host || !u_host) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->host_only) return fail(FGT_ERR_STATE, "host-only plan cannot execute");
  const size_t n = (size_t)plan->n_leaves * plan->np(), nu = (size_t)plan->n_targets() * plan->np();
  if (plan->stage && plan->stage_elems < n + nu) {
    cudaFree(plan->stage);
    plan->stage = nullptr;
  }
  if (!plan->stage) {
    cudaError_t e = cudaMalloc(&plan->stage, sizeof(double) * (n + nu));
    if (e != cudaSuccess) { plan->stage = nullptr; cudaGetLastError(); return fail(FGT_ERR_OOM, "staging buffers"); }
    plan->stage_elems = n + nu;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *sd = plan->stage, *ud = plan->stage + n;
  cudaError_t e = cudaMemcpyAsync(sd, sigma_host, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy in");
  fgt_status s = fgt_execute_async(plan, sd, ud, stream);
  if (s != FGT_OK) return s;
  e = cudaMemcpyAsync(u_host, ud, sizeof(double) * nu, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy out");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "transform");
  return FGT_OK;
}

fgt_status fgt_execute_host_async(fgt_plan *plan, const double *sigma_host, double *u_host, void *stream) {
  if (!plan || !sigma_host || !u_host) return fail(FGT_ERR_ARG, "NULL argument");
  if (plan->host_only) return fail(FGT_ERR_STATE, "host-only plan cannot execute");
  const size_t n = (size_t)plan->n_leaves * plan->np(), nu = (size_t)plan->n_targets() * plan->np();
  cudaError_t e = cudaSuccess;
  if (plan->hp_stage && plan->hp_elems < n + nu) {
    if ((e = cudaStreamSynchronize(plan->hp_out)) != cudaSuccess) return cuda_fail(e, "host pipeline");
    cudaFree(plan->hp_stage);
    plan->hp_stage = nullptr;
    plan->hp_used[0] = plan->hp_used[1] = false;
  }
  if (!plan->hp_in) {
    if (cudaStreamCreateWithFlags(&plan->hp_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&plan->hp_out, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return fail(FGT_ERR_OOM, "host pipeline streams");
    }
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&plan->hp_in_ev[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&plan->hp_done_ev[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&plan->hp_free_ev[i], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(FGT_ERR_OOM, "host pipeline events");
      }
  }
  if (!plan->hp_stage) {
    e = cudaMalloc(&plan->hp_stage, 2 * sizeof(double) * (n + nu));
    if (e != cudaSuccess) { plan->hp_stage = nullptr; cudaGetLastError(); return fail(FGT_ERR_OOM, "staging buffers"); }
    plan->hp_elems = n + nu;
  }
  const int slot = plan->hp_next;
  plan->hp_next ^= 1;
  cudaStream_t st = (cudaStream_t)stream;
  double *sd = plan->hp_stage + (size_t)slot * plan->hp_elems, *ud = sd + n;
  // copy in, once the call that last used this slot has copied its result out
  if (plan->hp_used[slot] && (e = cudaStreamWaitEvent(plan->hp_in, plan->hp_free_ev[slot], 0)) != cudaSuccess)
    return cuda_fail(e, "host pipeline");
  if ((e = cudaMemcpyAsync(sd, sigma_host, sizeof(double) * n, cudaMemcpyHostToDevice, plan->hp_in)) != cudaSuccess)
    return cuda_fail(e, "copy in");
  if ((e = cudaEventRecord(plan->hp_in_ev[slot], plan->hp_in)) != cudaSuccess) return cuda_fail(e, "host pipeline");
  // transform on the caller's stream once the input is there
  if ((e = cudaStreamWaitEvent(st, plan->hp_in_ev[slot], 0)) != cudaSuccess) return cuda_fail(e, "host pipeline");
  fgt_status s = fgt_execute_async(plan, sd, ud, stream);
  if (s != FGT_OK) return s;
  if ((e = cudaEventRecord(plan->hp_done_ev[slot], st)) != cudaSuccess) return cuda_fail(e, "host pipeline");
  // copy out on the copy-out stream, then free the slot
  if ((e = cudaStreamWaitEvent(plan->hp_out, plan->hp_done_ev[slot], 0)) != cudaSuccess)
    return cuda_fail(e, "host pipeline");
  if ((e = cudaMemcpyAsync(u_host, ud, sizeof(double) * nu, cudaMemcpyDeviceToHost, plan->hp_out)) != cudaSuccess)
    return cuda_fail(e, "copy out");
  if ((e = cudaEventRecord(plan->hp_free_ev[slot], plan->hp_out)) != cudaSuccess) return cuda_fail(e, "host pipeline");
  plan->hp_used[slot] = true;
  return FGT_OK;
}

fgt_status fgt_host_sync(fgt_plan *plan) {
  if (!plan) return fail(FGT_ERR_ARG, "NULL plan");
  if (!plan->hp_out) return FGT_OK;
  const cudaError_t e = cudaStreamSynchronize(plan->hp_out);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "host pipeline");
}

void fgt_destroy(fgt_plan *plan) { delete plan; }

const char *fgt_last_error(void) { return g_err.c_str(); }

fgt_status fgt_selftest_tc_timeout(void) {
  const cudaError_t e = fgt::selftest_tc_timeout();
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "time-out self-test");
}

fgt_status fgt_check_status(unsigned *site, unsigned *count, int *checked) {
  if (!site || !count || !checked) return fail(FGT_ERR_ARG, "NULL argument");
  const cudaError_t e = fgt::read_check(site, count, checked);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "check status");
}

fgt_status fgt_device_status(int *status) {
  if (!status) return fail(FGT_ERR_ARG, "status is NULL");
  const cudaError_t e = fgt::read_tc_status(status);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "device status");
}

fgt_status fgt_gauss_legendre(int k, double *nodes, double *weights) {
  if (k < 1 || k > 64 || !nodes || !weights) return fail(FGT_ERR_ARG, "k must be in [1, 64]");
  fgt::gl_rule(k, nodes, weights);
  return FGT_OK;
}

fgt_status fgt_params(double delta, double eps, int bc, int32_t *cutoff_level, double *D0, double *R, double *h,
                      int32_t *n_f, int32_t *n_p) {
  if (!(delta > 0) || !(eps > 0 && eps < 1)) return fail(FGT_ERR_ARG, "bad delta or eps");
  int lc, M, np, fourier;
  double d0, r, hh;
  choose_params(delta, eps, bc, lc, d0, r, hh, M, np, fourier);
  if (cutoff_level) *cutoff_level = lc;
  if (D0) *D0 = d0;
  if (R) *R = r;
  if (h) *h = hh;
  if (n_f) *n_f = 2 * M;
  if (n_p) *n_p = np;
  return FGT_OK;
}

int32_t fgt_nf_for_range(double eps, double R) {
  const double D0 = std::sqrt(std::log(3.0 / eps));
  return 2 * (int32_t)std::ceil(D0 * (R + D0) / kPi);
}

fgt_status fgt_legendre_gauss_integrals(double lambda, double t, int nmax, double *out) {
  if (!(lambda > 0) || nmax < 0 || nmax > 70 || !out) return fail(FGT_ERR_ARG, "bad argument");
  fgt::gauss_legendre_integrals(lambda, t, nmax, out);
  return FGT_OK;
}

fgt_status fgt_spherical_bessel(double x, int nmax, double *out) {
  if (nmax < 0 || nmax > 70 || !out || !std::isfinite(x) || std::fabs(x) > 1e4)
    return fail(FGT_ERR_ARG, "bad argument");
  fgt::spherical_bessel(x, nmax, out);
  return FGT_OK;
}

fgt_status fgt_legendre_fourier_integrals(double t, int nmax, double *re, double *im) {
  if (nmax < 0 || nmax > 70 || !re || !im || !std::isfinite(t) || std::fabs(t) > 1e4)
    return fail(FGT_ERR_ARG, "bad argument");
  fgt::legendre_fourier_integrals(t, nmax, re, im);
  return FGT_OK;
}

}  // extern "C"

// ============================================================================ batched execution
//
// Many independent transforms in one launch: the kernel sequence of every plan is captured
// once into a CUDA graph in which each transform is a branch (branches rotate over a small pool of
// capture streams, which chains the branches sharing one), so the device runs up to that many
// transforms concurrently and
// the host issues a single graph launch.  The graph is rebuilt only when the input / output
// pointers change.

struct fgt_batch {
  int mode = FGT_BATCH_GRAPH;
  fgt::BatchQueue *queue = nullptr;    // persistent mode: the device work queue
  std::vector<fgt_plan *> plans;
  std::vector<cudaStream_t> streams;   // branch streams used while capturing
  cudaStream_t cap = nullptr;          // capture origin
  std::vector<cudaEvent_t> events;     // [0] fork, [1..n] joins
  cudaGraphExec_t exec = nullptr;
  std::vector<const double *> sig;
  std::vector<double *> u;
  ~fgt_batch() {
    if (queue) fgt::batch_queue_destroy(queue);
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

fgt_status batch_capture(fgt_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(e, "batch capture");
  cudaError_t first = cudaEventRecord(b->events[0], b->cap);
  for (size_t i = 0; i < b->plans.size() && first == cudaSuccess; ++i) {
    cudaStream_t s = b->streams[i % b->streams.size()];
    first = cudaStreamWaitEvent(s, b->events[0], 0);
    if (first != cudaSuccess) break;
    fgt::ExecDesc ex = b->plans[i]->ex;
    ex.events = nullptr;
    first = fgt::run_transform(ex, b->sig[i], b->u[i], s);
    if (first != cudaSuccess) break;
    first = cudaEventRecord(b->events[1 + i], s);
    if (first != cudaSuccess) break;
    first = cudaStreamWaitEvent(b->cap, b->events[1 + i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  if (first != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return cuda_fail(first != cudaSuccess ? first : e, "batch capture");
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "batch graph instantiate");
  }
  return FGT_OK;
}

}  // namespace

extern "C" {

fgt_status fgt_batch_create(fgt_plan *const *plans, int n, fgt_batch **out) {
  return fgt_batch_create_mode(plans, n, FGT_BATCH_GRAPH, out);
}

fgt_status fgt_batch_create_mode(fgt_plan *const *plans, int n, int mode, fgt_batch **out) {
  if (!out || !plans || n < 1) return fail(FGT_ERR_ARG, "bad batch arguments");
  if (mode != FGT_BATCH_GRAPH && mode != FGT_BATCH_PERSISTENT) return fail(FGT_ERR_ARG, "bad batch mode");
  *out = nullptr;
  // every transform of the batch writes its plan's workspace and records its plan's side-stream
  // events: a plan listed twice would have two branches racing on them
  {
    std::unordered_set<const fgt_plan *> seen;
    for (int i = 0; i < n; ++i)
      if (plans[i] && !seen.insert(plans[i]).second)
        return fail(FGT_ERR_ARG, "batch plan " + std::to_string(i) + " is listed twice (duplicate plan pointer)");
  }
  fgt_batch *b = new (std::nothrow) fgt_batch();
  if (!b) return fail(FGT_ERR_OOM, "host allocation");
  for (int i = 0; i < n; ++i) {
    fgt_plan *p = plans[i];
    if (!p || p->host_only) { delete b; return fail(FGT_ERR_ARG, "batch plan " + std::to_string(i) + " is not a device plan"); }
    if (p->dirty) {
      fgt_status s = prepare(*p);
      if (s != FGT_OK) { delete b; return s; }
    }
    b->plans.push_back(p);
  }
  b->mode = mode;
  if (mode == FGT_BATCH_PERSISTENT) {
    std::vector<const fgt::ExecDesc *> ex;
    for (fgt_plan *p : b->plans) ex.push_back(&p->ex);
    const char *why = nullptr;
    cudaError_t ce = fgt::batch_queue_create(ex, &b->queue, &why);
    if (ce != cudaSuccess) { delete b; return cuda_fail(ce, "persistent batch queue"); }
    if (why) { delete b; return fail(FGT_ERR_ARG, std::string("persistent batch: a plan uses ") + why); }
    b->sig.assign(n, nullptr);
    b->u.assign(n, nullptr);
    *out = b;
    return FGT_OK;
  }
  // 16 capture streams: transforms sharing a stream are chained in the graph, so at most 16 run
  // at once; one stream per transform (every branch free) measured 1.9x slower on 256 transforms
  // (their working sets compete in L2)
  const int nstreams = std::min(n, 16);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int i = 0; i < nstreams && e == cudaSuccess; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
  }
  for (int i = 0; i <= n && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->events.push_back(ev);
  }
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "batch streams/events"); }
  b->sig.assign(n, nullptr);
  b->u.assign(n, nullptr);
  *out = b;
  return FGT_OK;
}

fgt_status fgt_batch_execute(fgt_batch *b, const double *const *sigma_dev, double *const *u_dev, void *stream) {
  if (!b || !sigma_dev || !u_dev) return fail(FGT_ERR_ARG, "NULL argument");
  bool same = b->exec != nullptr;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    if (!sigma_dev[i] || !u_dev[i]) return fail(FGT_ERR_ARG, "NULL buffer in batch");
    if (b->plans[i]->dirty) return fail(FGT_ERR_STATE, "a batch plan changed mode or precision; rebuild the batch");
    if (b->sig[i] != sigma_dev[i] || b->u[i] != u_dev[i]) same = false;
  }
  if (b->mode == FGT_BATCH_PERSISTENT) {
    cudaError_t ce = fgt::set_check_ranges(nullptr, nullptr, 0, (cudaStream_t)stream);
    if (ce == cudaSuccess) ce = fgt::batch_queue_run(b->queue, sigma_dev, u_dev, (cudaStream_t)stream, 1LL << 31);
    if (ce != cudaSuccess) return cuda_fail(ce, "persistent batch launch");
    return FGT_OK;
  }
  if (!same) {
    for (size_t i = 0; i < b->plans.size(); ++i) {
      b->sig[i] = sigma_dev[i];
      b->u[i] = u_dev[i];
    }
    fgt_status s = batch_capture(b);
    if (s != FGT_OK) return s;
  }
  cudaError_t e = fgt::set_check_ranges(nullptr, nullptr, 0, (cudaStream_t)stream);  // checked build: no checks
  if (e != cudaSuccess) return cuda_fail(e, "check ranges");
  e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return FGT_OK;
}

void fgt_batch_destroy(fgt_batch *b) { delete b; }

fgt_status fgt_batch_status(fgt_batch *b, int *status) {
  if (!b || !status) return fail(FGT_ERR_ARG, "NULL argument");
  *status = 0;
  if (b->mode != FGT_BATCH_PERSISTENT) return FGT_OK;
  int word = 0;
  cudaError_t e = fgt::batch_queue_status(b->queue, &word);
  if (e != cudaSuccess) return cuda_fail(e, "batch status");
  *status = word ? FGT_ERR_TIMEOUT : 0;
  return FGT_OK;
}

fgt_status fgt_batch_get_info(const fgt_batch *b, int *mode, int64_t *items, int *grid) {
  if (!b) return fail(FGT_ERR_ARG, "NULL batch");
  if (mode) *mode = b->mode;
  if (items) *items = b->queue ? (int64_t)fgt::batch_queue_items(b->queue) : 0;
  if (grid) *grid = b->queue ? fgt::batch_queue_grid(b->queue) : 0;
  return FGT_OK;
}

fgt_status fgt_selftest_batch_timeout(int *status) {
  if (!status) return fail(FGT_ERR_ARG, "NULL argument");
  int word = 0;
  cudaError_t e = fgt::selftest_batch_timeout(&word);
  if (e != cudaSuccess) return cuda_fail(e, "batch time-out self-test");
  *status = word ? FGT_ERR_TIMEOUT : 0;
  return FGT_OK;
}

fgt_status fgt_execute_batch(fgt_plan *const *plans, const double *const *sigma_dev, double *const *u_dev, int n,
                             void *stream) {
  fgt_batch *b = nullptr;
  fgt_status s = fgt_batch_create(plans, n, &b);
  if (s != FGT_OK) return s;
  s = fgt_batch_execute(b, sigma_dev, u_dev, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  fgt_batch_destroy(b);
  if (s != FGT_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "batch");
  return FGT_OK;
}

}  // extern "C"

// ============================================================================ point FGT (Algorithm 2)
//
// The discrete transform u(x_i) = sum_j exp(-|x_i - y_j|^2/delta) q_j in free space.  Algorithm 1's
// tree is taken at its cutoff level only: the root is the bounding cube of all points enlarged to
// 2^l_c boxes of side D0 sqrt(delta) (the "cutoff length"), every nonempty box at that level is a
// leaf.  A box holding more than n_s sources is dense: its sources are replaced by a k_p^d proxy
// grid (the plane-wave form then runs in tensor-product form, as the paper's closing remark
// proposes in place of the NUFFT), its outgoing expansion reaches every colleague through the
// diagonal translation, and the incoming expansion is evaluated on the target box's proxy grid and
// interpolated to the targets.  Sources of sparse boxes reach their colleagues' targets directly.
// k_p is the smallest grid on which Lagrange interpolation reproduces the highest plane wave of the
// expansion to 5e-2 eps on the box.

struct fgt_point_plan {
  int d = 0, n_s = 0, kp = 0, M = 0, n1 = 0, nh = 0, lc = 0, prec = 0;
  double delta = 0, tol = 0, D0 = 0, Lc = 0, h = 0, kappa = 0;
  int64_t n_src = 0, n_tgt = 0, n_box = 0, n_dense = 0, n_in = 0, n_direct = 0;
  fgt::ProxyRule pr{};
  fgt::ExecDesc ex;
  fgt::PointTargets pt;
  void *dev = nullptr;     // lists, tables, sorted points
  void *work = nullptr;    // phi, psi, Q, U, q_sorted
  size_t dev_bytes = 0, work_bytes = 0;
  const int64_t *aseg = nullptr, *s_id = nullptr;
  int64_t n_aseg = 0;
  const double *s_local = nullptr;
  double *Q = nullptr, *U = nullptr, *q_sorted = nullptr;
  float *q32 = nullptr;
  ~fgt_point_plan() {
    if (dev) cudaFree(dev);
    if (work) cudaFree(work);
  }
};

namespace {

struct Packer {
  std::vector<unsigned char> buf;
  template <typename T>
  size_t add(const std::vector<T> &v) {
    const size_t off = (buf.size() + 255) & ~(size_t)255;
    buf.resize(off + sizeof(T) * v.size());
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), sizeof(T) * v.size());
    return off;
  }
};

// Smallest Gauss-Legendre grid on which Lagrange interpolation reproduces every plane wave of the
// expansion well enough: mode m (phase kappa m (Lc/2) s over a box, s in [-1, 1]) enters the
// expansion with the relative weight exp(-m^2 h^2 / 4), so its interpolation error times that
// weight must stay within tol.
int proxy_order(double kappa_half_L, double h, int M, double tol, fgt::ProxyRule &pr) {
  for (int n = 4; n <= fgt::kMaxProxy; ++n) {
    double x[fgt::kMaxProxy], wt[fgt::kMaxProxy];
    fgt::gl_rule(n, x, wt);
    double bw[fgt::kMaxProxy];
    for (int t = 0; t < n; ++t) {
      double p = 1.0;
      for (int m = 0; m < n; ++m)
        if (m != t) p *= (x[t] - x[m]);
      bw[t] = 1.0 / p;
    }
    double worst = 0.0;
    for (int m = 1; m < M && worst <= tol; ++m) {
      const double w = kappa_half_L * m, rel = std::exp(-0.25 * m * m * h * h);
      for (int q = 0; q <= 400; ++q) {
        const double s = -1.0 + 2.0 * q / 400.0;
        double num_r = 0.0, num_i = 0.0, den = 0.0;
        bool hit = false;
        for (int t = 0; t < n; ++t) {
          const double dx = s - x[t];
          if (dx == 0.0) { hit = true; break; }
          const double c = bw[t] / dx;
          num_r += c * std::cos(w * x[t]);
          num_i += c * std::sin(w * x[t]);
          den += c;
        }
        if (hit) continue;
        worst = std::max(worst, rel * std::hypot(num_r / den - std::cos(w * s), num_i / den - std::sin(w * s)));
      }
    }
    if (worst <= tol) {
      double bmax = 0.0;
      for (int t = 0; t < n; ++t) {
        pr.x[t] = x[t];
        pr.bw[t] = bw[t];
        bmax = std::max(bmax, std::fabs(bw[t]));
      }
      for (int t = 0; t < n; ++t) {
        pr.xf[t] = (float)x[t];
        pr.bwf[t] = (float)(bw[t] / bmax);
      }
      return n;
    }
  }
  return -1;
}

}  // namespace

fgt_status fgt_point_plan_create(int d, double delta, double tol, int64_t n_src, const double *src, int64_t n_tgt,
                                 const double *tgt, int n_s, int prec, fgt_point_plan **out) {
  if (!out) return fail(FGT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if ((d != 2 && d != 3) || !(delta > 0) || !(tol > 0 && tol < 1) || n_src < 0 || n_tgt < 0 || n_s < 1 ||
      (n_src > 0 && !src) || (n_tgt > 0 && !tgt))
    return fail(FGT_ERR_ARG, "point plan: bad arguments");
  if (prec != FGT_PREC_FP64 && prec != FGT_PREC_SPLIT)
    return fail(FGT_ERR_ARG, "point plan: precision must be FGT_PREC_FP64 or FGT_PREC_SPLIT");
  if (prec == FGT_PREC_SPLIT && tol < 1e-7) return fail(FGT_ERR_ARG, "split precision needs tol >= 1e-7");
  const bool split = prec == FGT_PREC_SPLIT;
  auto *P = new (std::nothrow) fgt_point_plan();
  if (!P) return fail(FGT_ERR_OOM, "host allocation");
  std::unique_ptr<fgt_point_plan> guard(P);
  P->d = d; P->delta = delta; P->tol = tol; P->n_s = n_s; P->n_src = n_src; P->n_tgt = n_tgt;
  // Theorem 1 for colleagues at the cutoff length: |x_a - y_a| <= 2 D0 sqrt(delta), R = 2 D0
  P->D0 = std::sqrt(std::log(3.0 / tol));
  P->Lc = P->D0 * std::sqrt(delta);
  const double R = 2.0 * P->D0;
  P->h = 2.0 * kPi / (R + P->D0);
  P->M = (int)std::ceil(P->D0 * (R + P->D0) / kPi);
  P->n1 = 2 * P->M - 1;
  P->nh = P->M;
  P->kappa = P->h / std::sqrt(delta);
  P->kp = proxy_order(P->kappa * 0.5 * P->Lc, P->h, P->M, 0.1 * tol, P->pr);
  if (P->kp < 0) return fail(FGT_ERR_ARG, "point plan: tolerance needs a proxy grid above 40 nodes per axis");
  if (split && P->kp > fgt::kMaxProxy32)
    return fail(FGT_ERR_ARG, "point plan: split precision needs a proxy grid of at most 30 nodes per axis");
  P->prec = prec;
  // root: the bounding cube of all points, 2^l_c cutoff boxes wide
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) { lo[a] = HUGE_VAL; hi[a] = -HUGE_VAL; }
  for (const auto &pts : {std::make_pair(src, n_src), std::make_pair(tgt, n_tgt)})
    for (int64_t i = 0; i < pts.second; ++i)
      for (int a = 0; a < d; ++a) {
        const double v = pts.first[i * d + a];
        if (!std::isfinite(v)) return fail(FGT_ERR_ARG, "point plan: non-finite coordinate");
        lo[a] = std::min(lo[a], v);
        hi[a] = std::max(hi[a], v);
      }
  if (n_src + n_tgt == 0)
    for (int a = 0; a < d; ++a) lo[a] = hi[a] = 0.0;
  double ext = 0.0, c0[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) { ext = std::max(ext, hi[a] - lo[a]); c0[a] = 0.5 * (lo[a] + hi[a]); }
  int lc = 0;
  while (std::ldexp(P->Lc, lc) < ext * (1.0 + 1e-12) + 1e-300 && lc < 20) ++lc;
  if (std::ldexp(P->Lc, lc) < ext) return fail(FGT_ERR_ARG, "point plan: more than 2^20 cutoff boxes per axis");
  P->lc = lc;
  const int64_t nb = (int64_t)1 << lc;
  const double L0 = std::ldexp(P->Lc, lc);
  double corner[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) corner[a] = c0[a] - 0.5 * L0;
  // box of every point, and the nonempty boxes
  std::unordered_map<uint64_t, int32_t> box_of;
  std::vector<std::array<int32_t, 3>> bc;
  auto box_index = [&](const double *x, std::array<int32_t, 3> &c) {
    for (int a = 0; a < 3; ++a) c[a] = 0;
    for (int a = 0; a < d; ++a) {
      int64_t v = (int64_t)std::floor((x[a] - corner[a]) / P->Lc);
      c[a] = (int32_t)std::min<int64_t>(std::max<int64_t>(v, 0), nb - 1);
    }
    const uint64_t key = box_key(lc, c.data());
    auto it = box_of.find(key);
    if (it != box_of.end()) return it->second;
    const int32_t id = (int32_t)bc.size();
    box_of.emplace(key, id);
    bc.push_back(c);
    return id;
  };
  std::vector<int32_t> sbox(n_src), tbox(n_tgt);
  std::array<int32_t, 3> c{};
  for (int64_t j = 0; j < n_src; ++j) sbox[j] = box_index(src + j * d, c);
  for (int64_t i = 0; i < n_tgt; ++i) tbox[i] = box_index(tgt + i * d, c);
  const int64_t nbox = (int64_t)bc.size();
  P->n_box = nbox;
  // sources and targets sorted by box (counting sort)
  std::vector<int64_t> sptr(nbox + 1, 0), tptr(nbox + 1, 0);
  for (int32_t b : sbox) sptr[b + 1]++;
  for (int32_t b : tbox) tptr[b + 1]++;
  for (int64_t b = 0; b < nbox; ++b) { sptr[b + 1] += sptr[b]; tptr[b + 1] += tptr[b]; }
  std::vector<int64_t> s_id(n_src), t_id(n_tgt), fill_s(sptr.begin(), sptr.end() - 1), fill_t(tptr.begin(), tptr.end() - 1);
  for (int64_t j = 0; j < n_src; ++j) s_id[fill_s[sbox[j]]++] = j;
  for (int64_t i = 0; i < n_tgt; ++i) t_id[fill_t[tbox[i]]++] = i;
  auto centre = [&](int64_t b, int a) { return corner[a] + (bc[b][a] + 0.5) * P->Lc; };
  std::vector<double> s_xyz(n_src * d), s_loc(n_src * d), t_xyz(n_tgt * d), t_loc(n_tgt * d);
  for (int64_t j = 0; j < n_src; ++j)
    for (int a = 0; a < d; ++a) {
      s_xyz[j * d + a] = src[s_id[j] * d + a];
      s_loc[j * d + a] = (s_xyz[j * d + a] - centre(sbox[s_id[j]], a)) / (0.5 * P->Lc);
    }
  for (int64_t i = 0; i < n_tgt; ++i)
    for (int a = 0; a < d; ++a) {
      t_xyz[i * d + a] = tgt[t_id[i] * d + a];
      t_loc[i * d + a] = (t_xyz[i * d + a] - centre(tbox[t_id[i]], a)) / (0.5 * P->Lc);
    }
  // dense boxes (outgoing slots): their sources are the runs [sptr[b], sptr[b+1]) of the box order
  std::vector<int32_t> dense_slot(nbox, -1);
  std::vector<int64_t> aseg;  // (dense slot, first, end) segments of at most kPointSeg sources
  for (int64_t b = 0; b < nbox; ++b)
    if (sptr[b + 1] - sptr[b] > n_s) {
      dense_slot[b] = (int32_t)P->n_dense++;
      for (int64_t j = sptr[b]; j < sptr[b + 1]; j += fgt::kPointSeg) {
        aseg.push_back(dense_slot[b]);
        aseg.push_back(j);
        aseg.push_back(std::min(j + fgt::kPointSeg, sptr[b + 1]));
      }
    }
  P->n_aseg = (int64_t)aseg.size() / 3;
  // neighbour lists: incoming boxes (targets with a dense colleague), gather sources by code,
  // direct source boxes (sparse colleagues with sources)
  int noff = 1;
  for (int a = 0; a < d; ++a) noff *= 3;
  std::vector<int32_t> in_row(nbox, -1), gdst, dbox, dcode;
  std::vector<int64_t> gptr(1, 0), dptr(1, 0);
  std::vector<fgt::GatherSrc> gsrc;
  for (int64_t b = 0; b < nbox; ++b) {
    const bool has_t = tptr[b + 1] > tptr[b];
    std::vector<fgt::GatherSrc> g;
    for (int oc = 0; oc < noff; ++oc) {
      std::array<int32_t, 3> q{};
      bool ok = true;
      int code = 0, mul = 1;
      for (int a = 0, r = oc; a < d; ++a, r /= 3) {
        const int o = r % 3 - 1;
        const int64_t v = bc[b][a] + o;
        if (v < 0 || v >= nb) { ok = false; break; }
        q[a] = (int32_t)v;
        code += (o + 1) * mul;
        mul *= 3;
      }
      if (!ok) continue;
      auto it = box_of.find(box_key(lc, q.data()));
      if (it == box_of.end()) continue;
      const int32_t s = it->second;
      if (sptr[s + 1] == sptr[s]) continue;
      if (dense_slot[s] >= 0) g.push_back(fgt::GatherSrc{dense_slot[s], code});
      else if (has_t) {
        dbox.push_back(s);
        dcode.push_back(code);
      }
    }
    if (has_t) dptr.push_back((int64_t)dbox.size());
    if (has_t && !g.empty()) {
      in_row[b] = (int32_t)P->n_in++;
      gdst.push_back(in_row[b]);
      gsrc.insert(gsrc.end(), g.begin(), g.end());
      gptr.push_back((int64_t)gsrc.size());
    }
  }
  P->n_direct = (int64_t)dbox.size();
  // target boxes (those with targets), in box order, and their segments of <= kPointSeg targets
  std::vector<int32_t> tb_in;
  std::vector<int64_t> tseg;
  for (int64_t b = 0; b < nbox; ++b)
    if (tptr[b + 1] > tptr[b]) {
      const int64_t tb = (int64_t)tb_in.size();
      tb_in.push_back(in_row[b]);
      for (int64_t i = tptr[b]; i < tptr[b + 1]; i += fgt::kPointSeg) {
        tseg.push_back(tb);
        tseg.push_back(i);
        tseg.push_back(std::min(i + fgt::kPointSeg, tptr[b + 1]));
      }
    }
  // plane-wave matrices of a box about its own centre: form F[a][t] = w_a exp(-i kappa m_a
  // (Lc/2) eta_t) (last axis m >= 0, factor 2 for m > 0), evaluation E[t][a] = exp(+i ...)
  const int kp = P->kp, n1 = P->n1, nh = P->nh, M = P->M;
  std::vector<double2> Ff((size_t)n1 * kp), Fh((size_t)nh * kp), Ef((size_t)kp * n1), Eh((size_t)kp * nh);
  for (int a = 0; a < n1; ++a) {
    const int m = a - (M - 1);
    const double w = P->h / (2.0 * std::sqrt(kPi)) * std::exp(-0.25 * m * m * P->h * P->h);
    for (int t = 0; t < kp; ++t) {
      const double ph = P->kappa * m * 0.5 * P->Lc * P->pr.x[t];
      Ff[(size_t)a * kp + t] = make_double2(w * std::cos(ph), -w * std::sin(ph));
      Ef[(size_t)t * n1 + a] = make_double2(std::cos(ph), std::sin(ph));
      if (m >= 0) {
        Fh[(size_t)m * kp + t] = make_double2((m == 0 ? 1.0 : 2.0) * w * std::cos(ph), -(m == 0 ? 1.0 : 2.0) * w * std::sin(ph));
        Eh[(size_t)t * nh + m] = make_double2(std::cos(ph), std::sin(ph));
      }
    }
  }
  // diagonal translation phases for S = T + o: exp(+i k (c_T - c_S)) = exp(-i kappa m o Lc)
  std::vector<double2> Pf((size_t)3 * n1), Ph((size_t)3 * nh);
  for (int o = -1; o <= 1; ++o) {
    for (int a = 0; a < n1; ++a) {
      const double ph = -P->kappa * (a - (M - 1)) * o * P->Lc;
      Pf[(size_t)(o + 1) * n1 + a] = make_double2(std::cos(ph), std::sin(ph));
    }
    for (int b = 0; b < nh; ++b) {
      const double ph = -P->kappa * b * o * P->Lc;
      Ph[(size_t)(o + 1) * nh + b] = make_double2(std::cos(ph), std::sin(ph));
    }
  }
  // form blocks (dense boxes) and evaluation blocks (incoming boxes): one proxy grid each
  std::vector<fgt::Block> fblk, eblk;
  std::vector<int64_t> fleaf, eleaf;
  for (int64_t i = 0; i < P->n_dense; ++i) {
    fgt::Block b{};
    b.slot = (int32_t)i; b.K = kp; b.dl = 0; b.flags = 0; b.leaf0 = (int64_t)fleaf.size();
    fleaf.push_back(i);
    fblk.push_back(b);
  }
  for (int64_t i = 0; i < P->n_in; ++i) {
    fgt::Block b{};
    b.slot = (int32_t)i; b.K = kp; b.dl = 0; b.flags = 0; b.leaf0 = (int64_t)eleaf.size();
    eleaf.push_back(i);
    eblk.push_back(b);
  }
  Packer pk;
  const size_t o_fblk = pk.add(fblk), o_eblk = pk.add(eblk), o_fleaf = pk.add(fleaf), o_eleaf = pk.add(eleaf);
  // complex tables in the expansions' precision
  auto add_c = [&](const std::vector<double2> &v) {
    if (!split) return pk.add(v);
    std::vector<float2> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = make_float2((float)v[i].x, (float)v[i].y);
    return pk.add(f);
  };
  const size_t o_Ff = add_c(Ff), o_Fh = add_c(Fh), o_Ef = add_c(Ef), o_Eh = add_c(Eh), o_Pf = add_c(Pf),
               o_Ph = add_c(Ph);
  const size_t o_gdst = pk.add(gdst), o_gptr = pk.add(gptr), o_gsrc = pk.add(gsrc);
  const size_t o_aseg = pk.add(aseg), o_sloc = pk.add(s_loc);
  const size_t o_tseg = pk.add(tseg), o_txyz = pk.add(t_xyz), o_tloc = pk.add(t_loc), o_tid = pk.add(t_id),
               o_tbin = pk.add(tb_in), o_dp = pk.add(dptr), o_db = pk.add(dbox), o_sp = pk.add(sptr),
               o_sxyz = pk.add(s_xyz), o_sid = pk.add(s_id), o_dcode = pk.add(dcode);
  std::vector<float> s_loc32;
  if (split) s_loc32.assign(s_loc.begin(), s_loc.end());
  const size_t o_sloc32 = pk.add(s_loc32);
  cudaError_t e = cudaMalloc(&P->dev, std::max<size_t>(pk.buf.size(), 256));
  P->dev_bytes = std::max<size_t>(pk.buf.size(), 256);
  if (e != cudaSuccess) { P->dev = nullptr; cudaGetLastError(); return fail(FGT_ERR_OOM, "point plan: device tables"); }
  e = cudaMemcpy(P->dev, pk.buf.data(), pk.buf.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "point plan upload");
  auto at = [&](size_t off) { return (const void *)((const char *)P->dev + off); };
  const int64_t np = d == 3 ? (int64_t)kp * kp * kp : (int64_t)kp * kp;
  const int64_t ss = d == 3 ? (int64_t)nh * n1 * n1 : (int64_t)nh * n1;
  const size_t csz = split ? sizeof(float2) : sizeof(double2);
  const size_t phi_b = csz * ss * P->n_dense, psi_b = csz * ss * P->n_in;
  const size_t q_b = sizeof(double) * np * P->n_dense, u_b = sizeof(double) * np * P->n_in;
  const size_t qs_b = sizeof(double) * std::max<int64_t>(n_src, 1);
  const size_t q32_b = split ? sizeof(float) * std::max<int64_t>(n_src, 1) : 0;
  size_t off = 0;
  auto place = [&](size_t bytes) { const size_t o = off; off = (off + bytes + 255) & ~(size_t)255; return o; };
  const size_t w_phi = place(phi_b), w_psi = place(psi_b), w_q = place(q_b), w_u = place(u_b), w_qs = place(qs_b),
               w_q32 = place(q32_b);
  e = cudaMalloc(&P->work, std::max<size_t>(off, 256));
  P->work_bytes = std::max<size_t>(off, 256);
  if (e != cudaSuccess) { P->work = nullptr; cudaGetLastError(); return fail(FGT_ERR_OOM, "point plan: workspace"); }
  auto wk = [&](size_t o) { return (void *)((char *)P->work + o); };
  P->Q = (double *)wk(w_q);
  P->U = (double *)wk(w_u);
  P->q_sorted = (double *)wk(w_qs);
  P->q32 = split ? (float *)wk(w_q32) : nullptr;
  P->aseg = (const int64_t *)at(o_aseg);
  P->s_local = (const double *)at(o_sloc);
  P->s_id = (const int64_t *)at(o_sid);
  fgt::ExecDesc &x = P->ex;
  x.d = d; x.k = kp; x.n1 = n1; x.nh = nh; x.prec = split ? 1 : 0; x.fourier = 0;
  x.slot_size = ss;
  x.n_phi_slots = P->n_dense; x.n_psi_slots = P->n_in;
  x.phi = wk(w_phi); x.psi = wk(w_psi);
  x.blocks = (const fgt::Block *)at(o_fblk);
  x.n_blocks = P->n_dense;
  x.Kmax = kp;
  x.f1_blocks = (const fgt::Block *)at(o_fblk);
  x.n_f1 = P->n_dense;
  x.Kmax_f1 = kp;
  x.e1_blocks = (const fgt::Block *)at(o_eblk);
  x.n_e1 = P->n_in;
  x.Kmax_e1 = kp;
  x.block_leaves = (const int64_t *)at(o_fleaf);
  x.eval_leaves = (const int64_t *)at(o_eleaf);
  x.Ff = at(o_Ff); x.Fh = at(o_Fh); x.Ef = at(o_Ef); x.Eh = at(o_Eh);
  x.n_gather = P->n_in;
  x.gather_dst = (const int32_t *)at(o_gdst);
  x.gather_ptr = (const int64_t *)at(o_gptr);
  x.gather_src = (const fgt::GatherSrc *)at(o_gsrc);
  x.Pf = at(o_Pf); x.Ph = at(o_Ph);
  x.n_points = P->n_in * np;
  fgt::PointTargets &t = P->pt;
  t.d = d; t.kp = kp; t.f32 = split ? 1 : 0; t.delta = delta;
  t.n_tseg = (int64_t)tseg.size() / 3;
  t.tseg = (const int64_t *)at(o_tseg);
  t.t_xyz = (const double *)at(o_txyz);
  t.t_local = (const double *)at(o_tloc);
  t.t_id = (const int64_t *)at(o_tid);
  t.tbox_in = (const int32_t *)at(o_tbin);
  t.U = P->U;
  t.dptr = (const int64_t *)at(o_dp);
  t.dbox = (const int32_t *)at(o_db);
  t.sptr = (const int64_t *)at(o_sp);
  t.s_xyz = (const double *)at(o_sxyz);
  t.q_sorted = P->q_sorted;
  t.inv_delta = 1.0 / delta;
  t.dcode = (const int32_t *)at(o_dcode);
  t.s_local32 = split ? (const float *)at(o_sloc32) : nullptr;
  t.q32 = P->q32;
  t.dcoef = (float)(0.25 * P->Lc * P->Lc / delta);
  *out = guard.release();
  return FGT_OK;
}

fgt_status fgt_point_execute(fgt_point_plan *P, const double *q_dev, double *u_dev, void *stream) {
  if (!P || (P->n_src > 0 && !q_dev) || (P->n_tgt > 0 && !u_dev)) return fail(FGT_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  {  // checked build: q, u, the plan's tables and workspace
    const void *b[4] = {q_dev, u_dev, P->dev, P->work};
    const size_t n[4] = {8 * (size_t)P->n_src, 8 * (size_t)P->n_tgt, P->dev_bytes, P->work_bytes};
    cudaError_t ce = fgt::set_check_ranges(b, n, 4, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "check ranges");
  }
  cudaError_t e = fgt::point_gather_q(P->n_src, P->s_id, q_dev, P->q_sorted, P->q32, st);
  if (e == cudaSuccess)
    e = fgt::point_anterp(P->d, P->kp, P->prec == FGT_PREC_SPLIT, P->pr, P->n_dense, P->n_aseg, P->aseg,
                          P->s_local, P->q_sorted, P->Q, st);
  if (e == cudaSuccess && P->n_dense > 0 && P->n_in > 0) e = fgt::run_transform(P->ex, P->Q, P->U, st);
  if (e == cudaSuccess) e = fgt::point_targets(P->pt, P->pr, u_dev, st);
  return e == cudaSuccess ? FGT_OK : cuda_fail(e, "point transform");
}

fgt_status fgt_point_plan_get_info(const fgt_point_plan *P, fgt_point_info *info) {
  if (!P || !info) return fail(FGT_ERR_ARG, "NULL argument");
  info->cutoff_level = P->lc;
  info->proxy_order = P->kp;
  info->modes_1d = P->n1;
  info->n_boxes = P->n_box;
  info->n_dense_boxes = P->n_dense;
  info->n_incoming_boxes = P->n_in;
  info->n_direct_pairs = P->n_direct;
  info->cutoff_length = P->Lc;
  info->prec = P->prec;
  return FGT_OK;
}

void fgt_point_destroy(fgt_point_plan *P) { delete P; }
