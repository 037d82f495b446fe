/*
 * CPU FP64 oracle for the continuous ("box") Gauss transform — TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file's library.  It shares no code with the GPU path.
 *
 * What it computes (paper, Section 1, eq. (bgt) with kernels (gkernel) and
 * (gper_kernel)):
 *
 *     u(x) = \int_B G(x - y; delta) sigma~(y) dy,   B = [-1/2, 1/2]^d,
 *
 * at every tensor-product Gauss-Legendre node x of the requested target
 * leaves.  sigma~ is the density the box FGT actually transforms: on each leaf
 * S it is the degree-(p-1) tensor Lagrange interpolant of the p^d node values
 * (Section 2.4, eq. (papprox): a degree < p Legendre expansion determined by
 * values at p Gauss nodes is that same interpolant).
 *
 * G is separable, G(x) = prod_i g(x_i) (free: g(t) = exp(-t^2/delta);
 * periodic: g(t) = sum_n exp(-(t+n)^2/delta)), and sigma~ is a tensor product
 * of 1D Lagrange bases on each leaf, so the contribution of one source leaf S
 * to one target leaf T is a triple (double) product of 1D matrices
 *
 *     K_i[t][j] = \int_{S_i} g(x_t - y) l^S_j(y) dy ,
 *
 * applied dimension by dimension.  Each K_i entry is integrated with
 * composite Gauss-Legendre quadrature: the integration interval is cut to
 * where the Gaussian exceeds 1e-18 (for the periodic kernel: per image n,
 * images summed in order of increasing |n| while any part lies within that
 * range), split into panels no wider than sqrt(delta)/2 (nor wider than the
 * leaf), with max(24, p+16) nodes per panel.  The Lagrange basis is evaluated
 * from its product definition.  Source leaves farther than the 1e-18 range
 * (box-to-box distance, minimum image for the periodic kernel) contribute
 * nothing and are skipped.  The sum over source leaves is compensated
 * (Neumaier), so the result does not depend on the visiting order beyond
 * rounding.
 *
 * It uses none of the paper's machinery (no plane waves, no recurrences, no
 * tables, no lists): it is the defining integral, evaluated directly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define ORC_MAXP 32
#define ORC_CUT 1e-18

/* ---------- Gauss-Legendre rule on [-1,1] by Newton iteration on P_n ---------- */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; i++) {
    /* initial guess (Tricomi), ascending order after the sign flip below */
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z); P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1) */
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        /* one more step for full accuracy */
        p0 = 1.0; p1 = z;
        for (int k = 2; k <= n; k++) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1; p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
      x[n - 1 - i] = z;
      w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
}

/* ---------- Lagrange basis through the p nodes eta, evaluated at s ---------- */
static void lagrange_all(int p, const double *eta, double s, double *out) {
  for (int j = 0; j < p; j++) {
    double v = 1.0;
    for (int m = 0; m < p; m++)
      if (m != j) v *= (s - eta[m]) / (eta[j] - eta[m]);
    out[j] = v;
  }
}

typedef struct {
  int d, p, periodic;
  double delta, rcut;           /* rcut: exp(-rcut^2/delta) = 1e-18 */
  int nq;                        /* quadrature nodes per panel */
  double eta[ORC_MAXP], weta[ORC_MAXP];
  double xq[64], wq[64];
  long n_leaves;
  const int *level, *coord;
  const double *sigma;
  long n_targets;
  const long *targets;           /* target leaves of the source tree, or */
  const int *tlevel, *tcoord;    /* target boxes of their own (tlevel != NULL) */
  double *u;
  long next;                     /* work counter (guarded by mtx) */
  pthread_mutex_t mtx;
  int err;
} orc_ctx;

/* \int_a^b exp(-(x - y + shift)^2/delta) l_j((y - c) 2/L) dy for all j, added into acc[j].
 * Integration restricted to the part of [a,b] where the Gaussian exceeds the cutoff. */
static void add_1d_integral(const orc_ctx *C, double x, double shift, double a, double b,
                            double c, double L, double *acc) {
  double lo = x + shift - C->rcut, hi = x + shift + C->rcut;
  if (lo < a) lo = a;
  if (hi > b) hi = b;
  if (!(hi > lo)) return;
  double pw = 0.5 * sqrt(C->delta);
  if (pw > L) pw = L;
  int npan = (int)ceil((hi - lo) / pw);
  if (npan < 1) npan = 1;
  double hpan = (hi - lo) / npan;
  double lj[ORC_MAXP];
  for (int q = 0; q < npan; q++) {
    double pa = lo + q * hpan;
    for (int r = 0; r < C->nq; r++) {
      double y = pa + 0.5 * hpan * (C->xq[r] + 1.0);
      double wy = 0.5 * hpan * C->wq[r];
      double t = x - y + shift;
      double g = exp(-t * t / C->delta) * wy;
      lagrange_all(C->p, C->eta, (y - c) * 2.0 / L, lj);
      for (int j = 0; j < C->p; j++) acc[j] += g * lj[j];
    }
  }
}

/* K[t][j] for target nodes x_t = ct + (Lt/2) eta_t, source interval centred cs, side Ls. */
static void kernel_matrix(const orc_ctx *C, double ct, double Lt, double cs, double Ls, double *K) {
  int p = C->p;
  double a = cs - 0.5 * Ls, b = cs + 0.5 * Ls;
  for (int t = 0; t < p; t++) {
    double x = ct + 0.5 * Lt * C->eta[t];
    double acc[ORC_MAXP];
    for (int j = 0; j < p; j++) acc[j] = 0.0;
    if (!C->periodic) {
      add_1d_integral(C, x, 0.0, a, b, cs, Ls, acc);
    } else {
      /* images y -> y - n, i.e. g_p(x - y) = sum_n exp(-(x - y + n)^2/delta);
       * |x - y| <= 1, so images with |n| > rcut + 1 are below the cutoff everywhere */
      int nmax = (int)ceil(C->rcut) + 1;
      for (int n = 0; n <= nmax; n++) {
        add_1d_integral(C, x, (double)n, a, b, cs, Ls, acc);
        if (n) add_1d_integral(C, x, (double)-n, a, b, cs, Ls, acc);
      }
    }
    for (int j = 0; j < p; j++) K[t * p + j] = acc[j];
  }
}

static double box_center(int level, int c) { return -0.5 + (c + 0.5) * ldexp(1.0, -level); }

/* per-target cache of 1D matrices keyed by (source level, source coordinate) in one dimension */
typedef struct { int lev, crd; double *K; } kcache_ent;
typedef struct { kcache_ent *e; int n, cap; } kcache;

static const double *kcache_get(const orc_ctx *C, kcache *kc, double ct, double Lt, int slev, int scrd) {
  for (int i = 0; i < kc->n; i++)
    if (kc->e[i].lev == slev && kc->e[i].crd == scrd) return kc->e[i].K;
  if (kc->n == kc->cap) {
    int nc = kc->cap ? 2 * kc->cap : 64;
    kcache_ent *ne = (kcache_ent *)realloc(kc->e, sizeof(kcache_ent) * nc);
    if (!ne) return NULL;
    kc->e = ne; kc->cap = nc;
  }
  double *K = (double *)malloc(sizeof(double) * C->p * C->p);
  if (!K) return NULL;
  kernel_matrix(C, ct, Lt, box_center(slev, scrd), ldexp(1.0, -slev), K);
  kc->e[kc->n].lev = slev; kc->e[kc->n].crd = scrd; kc->e[kc->n].K = K;
  kc->n++;
  return K;
}

static void kcache_clear(kcache *kc) {
  for (int i = 0; i < kc->n; i++) free(kc->e[i].K);
  kc->n = 0;
}

/* squared distance between a target box (level lt, coordinates tc) and source leaf S (minimum
 * image when periodic) */
static double box_dist2(const orc_ctx *C, int lt, const int *tc, long S) {
  double d2 = 0.0;
  for (int i = 0; i < C->d; i++) {
    int ls = C->level[S];
    double ct = box_center(lt, tc[i]);
    double cs = box_center(ls, C->coord[S * C->d + i]);
    double half = 0.5 * (ldexp(1.0, -lt) + ldexp(1.0, -ls));
    double dc = fabs(ct - cs);
    if (C->periodic) dc = fmin(dc, fabs(1.0 - dc));
    double gap = dc - half;
    if (gap > 0) d2 += gap * gap;
  }
  return d2;
}

static void one_target(orc_ctx *C, long ti, kcache kc[3], double *work) {
  int d = C->d, p = C->p;
  int lt;
  const int *tc;
  if (C->tlevel) {
    lt = C->tlevel[ti];
    tc = C->tcoord + ti * C->d;
  } else {
    lt = C->level[C->targets[ti]];
    tc = C->coord + C->targets[ti] * C->d;
  }
  int np = 1;
  for (int i = 0; i < d; i++) np *= p;
  double *sum = work, *comp = work + np, *A = work + 2 * np, *Bm = work + 3 * np, *Cm = work + 4 * np;
  for (int q = 0; q < np; q++) { sum[q] = 0.0; comp[q] = 0.0; }
  double Lt = ldexp(1.0, -lt);
  double r2 = C->delta * log(1.0 / ORC_CUT);
  for (int i = 0; i < d; i++) kcache_clear(&kc[i]);
  for (long S = 0; S < C->n_leaves; S++) {
    if (box_dist2(C, lt, tc, S) > r2) continue;
    const double *K[3] = {NULL, NULL, NULL};
    for (int i = 0; i < d; i++) {
      K[i] = kcache_get(C, &kc[i], box_center(lt, tc[i]), Lt, C->level[S], C->coord[S * d + i]);
      if (!K[i]) { C->err = 1; return; }
    }
    const double *sg = C->sigma + S * np;
    /* contribution c = (K_d x ... x K_1) sigma_S, applied one dimension at a time;
       node index j_1 (x_1) fastest */
    if (d == 2) {
      /* A[j2][t1] = sum_j1 K1[t1][j1] s[j2][j1];  C[t2][t1] = sum_j2 K2[t2][j2] A[j2][t1] */
      for (int j2 = 0; j2 < p; j2++)
        for (int t1 = 0; t1 < p; t1++) {
          double a = 0.0;
          for (int j1 = 0; j1 < p; j1++) a += K[0][t1 * p + j1] * sg[j2 * p + j1];
          A[j2 * p + t1] = a;
        }
      for (int t2 = 0; t2 < p; t2++)
        for (int t1 = 0; t1 < p; t1++) {
          double a = 0.0;
          for (int j2 = 0; j2 < p; j2++) a += K[1][t2 * p + j2] * A[j2 * p + t1];
          Cm[t2 * p + t1] = a;
        }
    } else {
      for (int j3 = 0; j3 < p; j3++)
        for (int j2 = 0; j2 < p; j2++)
          for (int t1 = 0; t1 < p; t1++) {
            double a = 0.0;
            for (int j1 = 0; j1 < p; j1++) a += K[0][t1 * p + j1] * sg[(j3 * p + j2) * p + j1];
            A[(j3 * p + j2) * p + t1] = a;
          }
      for (int j3 = 0; j3 < p; j3++)
        for (int t2 = 0; t2 < p; t2++)
          for (int t1 = 0; t1 < p; t1++) {
            double a = 0.0;
            for (int j2 = 0; j2 < p; j2++) a += K[1][t2 * p + j2] * A[(j3 * p + j2) * p + t1];
            Bm[(j3 * p + t2) * p + t1] = a;
          }
      for (int t3 = 0; t3 < p; t3++)
        for (int t2 = 0; t2 < p; t2++)
          for (int t1 = 0; t1 < p; t1++) {
            double a = 0.0;
            for (int j3 = 0; j3 < p; j3++) a += K[2][t3 * p + j3] * Bm[(j3 * p + t2) * p + t1];
            Cm[(t3 * p + t2) * p + t1] = a;
          }
    }
    /* Neumaier compensated accumulation over source leaves */
    for (int q = 0; q < np; q++) {
      double s = sum[q], v = Cm[q], t = s + v;
      if (fabs(s) >= fabs(v)) comp[q] += (s - t) + v; else comp[q] += (v - t) + s;
      sum[q] = t;
    }
  }
  double *uo = C->u + ti * np;
  for (int q = 0; q < np; q++) uo[q] = sum[q] + comp[q];
}

static void *worker(void *arg) {
  orc_ctx *C = (orc_ctx *)arg;
  int np = 1;
  for (int i = 0; i < C->d; i++) np *= C->p;
  double *work = (double *)malloc(sizeof(double) * 5 * np);
  kcache kc[3];
  memset(kc, 0, sizeof(kc));
  if (!work) { C->err = 1; return NULL; }
  for (;;) {
    pthread_mutex_lock(&C->mtx);
    long ti = C->next++;
    pthread_mutex_unlock(&C->mtx);
    if (ti >= C->n_targets || C->err) break;
    one_target(C, ti, kc, work);
  }
  for (int i = 0; i < 3; i++) { kcache_clear(&kc[i]); free(kc[i].e); }
  free(work);
  return NULL;
}

/* Number of threads the oracle uses when asked for 0 (all online cores). */
int oracle_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/*
 * u at the nodes of the target leaves targets[0..n_targets).
 * leaf_level[n_leaves], leaf_coord[n_leaves*d] (integer box index at its level),
 * sigma[n_leaves][p^d] with node index j_1 fastest; u_out[n_targets][p^d].
 * Returns 0 on success, nonzero on bad arguments or allocation failure.
 */
int oracle_box_fgt(int d, int p, double delta, int periodic, long n_leaves,
                   const int *leaf_level, const int *leaf_coord, const double *sigma,
                   long n_targets, const long *targets, double *u_out, int n_threads) {
  if ((d != 2 && d != 3) || p < 1 || p > ORC_MAXP || !(delta > 0) || n_leaves < 0 || n_targets < 0)
    return 1;
  orc_ctx C;
  memset(&C, 0, sizeof(C));
  C.d = d; C.p = p; C.periodic = periodic ? 1 : 0; C.delta = delta;
  C.rcut = sqrt(delta * log(1.0 / ORC_CUT));
  C.nq = p + 16 > 24 ? p + 16 : 24;
  gauss_legendre(p, C.eta, C.weta);
  gauss_legendre(C.nq, C.xq, C.wq);
  C.n_leaves = n_leaves; C.level = leaf_level; C.coord = leaf_coord; C.sigma = sigma;
  C.n_targets = n_targets; C.targets = targets; C.u = u_out;
  for (long t = 0; t < n_targets; t++)
    if (targets[t] < 0 || targets[t] >= n_leaves) return 1;
  pthread_mutex_init(&C.mtx, NULL);
  int nt = n_threads > 0 ? n_threads : oracle_default_threads();
  if (nt > 256) nt = 256;
  pthread_t th[256];
  int started = 0;
  for (int i = 0; i < nt; i++)
    if (pthread_create(&th[i], NULL, worker, &C) == 0) started++; else break;
  if (started == 0) worker(&C);
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&C.mtx);
  return C.err;
}

/*
 * u at the nodes of target boxes of their own: box t has level tgt_level[t] and integer
 * coordinates tgt_coord[t*d .. t*d+d) (any level, 0 <= coordinate < 2^level), its nodes laid out
 * like a leaf's.  Used for output trees that refine or coarsen the source tree (Algorithms 5, 6).
 */
int oracle_box_fgt_boxes(int d, int p, double delta, int periodic, long n_leaves,
                         const int *leaf_level, const int *leaf_coord, const double *sigma,
                         long n_tboxes, const int *tgt_level, const int *tgt_coord, double *u_out, int n_threads) {
  if ((d != 2 && d != 3) || p < 1 || p > ORC_MAXP || !(delta > 0) || n_leaves < 0 || n_tboxes < 0)
    return 1;
  for (long t = 0; t < n_tboxes; t++) {
    if (tgt_level[t] < 0 || tgt_level[t] > 30) return 1;
    for (int i = 0; i < d; i++)
      if (tgt_coord[t * d + i] < 0 || tgt_coord[t * d + i] >= (1 << tgt_level[t])) return 1;
  }
  orc_ctx C;
  memset(&C, 0, sizeof(C));
  C.d = d; C.p = p; C.periodic = periodic ? 1 : 0; C.delta = delta;
  C.rcut = sqrt(delta * log(1.0 / ORC_CUT));
  C.nq = p + 16 > 24 ? p + 16 : 24;
  gauss_legendre(p, C.eta, C.weta);
  gauss_legendre(C.nq, C.xq, C.wq);
  C.n_leaves = n_leaves; C.level = leaf_level; C.coord = leaf_coord; C.sigma = sigma;
  C.n_targets = n_tboxes; C.tlevel = tgt_level; C.tcoord = tgt_coord; C.u = u_out;
  pthread_mutex_init(&C.mtx, NULL);
  int nt = n_threads > 0 ? n_threads : oracle_default_threads();
  if (nt > 256) nt = 256;
  pthread_t th[256];
  int started = 0;
  for (int i = 0; i < nt; i++)
    if (pthread_create(&th[i], NULL, worker, &C) == 0) started++; else break;
  if (started == 0) worker(&C);
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&C.mtx);
  return C.err;
}

/* ---- discrete Gauss transform (Section 3's point FGT): the definition summed directly ---- */

typedef struct {
  int d;
  double delta;
  long n_src, n_tgt;
  const double *src, *q, *tgt;
  double *u;
  long next;
  pthread_mutex_t mtx;
} pt_ctx;

static void *pt_worker(void *arg) {
  pt_ctx *C = (pt_ctx *)arg;
  for (;;) {
    pthread_mutex_lock(&C->mtx);
    long i0 = C->next;
    C->next += 256;
    pthread_mutex_unlock(&C->mtx);
    if (i0 >= C->n_tgt) break;
    long i1 = i0 + 256 < C->n_tgt ? i0 + 256 : C->n_tgt;
    for (long i = i0; i < i1; i++) {
      const double *x = C->tgt + i * C->d;
      double sum = 0.0, comp = 0.0;
      for (long j = 0; j < C->n_src; j++) {
        const double *y = C->src + j * C->d;
        double r2 = 0.0;
        for (int a = 0; a < C->d; a++) r2 += (x[a] - y[a]) * (x[a] - y[a]);
        double v = exp(-r2 / C->delta) * C->q[j];
        double t = sum + v;   /* Neumaier compensated sum */
        if (fabs(sum) >= fabs(v)) comp += (sum - t) + v; else comp += (v - t) + sum;
        sum = t;
      }
      C->u[i] = sum + comp;
    }
  }
  return NULL;
}

/*
 * u[i] = sum_j exp(-|x_i - y_j|^2 / delta) q_j for n_tgt targets x (tgt[n_tgt][d]) and n_src
 * sources y (src[n_src][d]) with weights q, free space.  O(n_tgt n_src), all pairs, no cutoff.
 */
int oracle_point_fgt(int d, double delta, long n_src, const double *src, const double *q, long n_tgt,
                     const double *tgt, double *u_out, int n_threads) {
  if ((d != 1 && d != 2 && d != 3) || !(delta > 0) || n_src < 0 || n_tgt < 0) return 1;
  pt_ctx C;
  memset(&C, 0, sizeof(C));
  C.d = d; C.delta = delta; C.n_src = n_src; C.n_tgt = n_tgt; C.src = src; C.q = q; C.tgt = tgt; C.u = u_out;
  pthread_mutex_init(&C.mtx, NULL);
  int nt = n_threads > 0 ? n_threads : oracle_default_threads();
  if (nt > 256) nt = 256;
  pthread_t th[256];
  int started = 0;
  for (int i = 0; i < nt; i++)
    if (pthread_create(&th[i], NULL, pt_worker, &C) == 0) started++; else break;
  if (started == 0) pt_worker(&C);
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&C.mtx);
  return 0;
}

/* The oracle's own Gauss-Legendre rule (exported so the tests can pin it). */
int oracle_gauss_legendre(int n, double *x, double *w) {
  if (n < 1 || n > 64) return 1;
  gauss_legendre(n, x, w);
  return 0;
}
