// CUDA kernels of the box FGT (Algorithm 4, Section 4.2) for sm_103a.
//
//   form_kernel    outgoing plane-wave expansion of a dense block of leaves,
//                  three (two in 2D) successive 1D contractions (Lemma pwbox,
//                  Remark pwcost), accumulated into its anchor's slot.
//   merge_kernel   child -> parent diagonal shift T_c->p (hierarchical mode).
//   gather_kernel  out -> in diagonal translation T_out->in at the cutoff level,
//                  eq. (diagonaltranslation).
//   push_kernel    parent -> child diagonal shift T_p->c (hierarchical mode).
//   eval_kernel    incoming expansion -> tensor grid of a dense block
//                  (Lemma thm:pweval), real part.
//   near_kernel    D-list interactions through separable k x k tables
//                  (Lemma directbox, Remark dircost, Definitions pol2potdef*).
//
// Expansion slots hold n1^(d-1) * nh complex coefficients: axes 1..d-1 carry
// the full symmetric mode range, the last axis only m >= 0 (conjugate
// symmetry of a real density; the factor 2 of the m > 0 modes is folded into
// the form matrices).  Slot index: ((m_3 * n1) + m_2) * n1 + m_1 in 3D and
// m_2 * n1 + m_1 in 2D, m_1 fastest.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "fgt_exec.h"

namespace fgt {

template <typename R> struct C2T;
template <> struct C2T<double> { using T = double2; };
template <> struct C2T<float> { using T = float2; };

template <typename R, typename C>
__device__ __forceinline__ void cfma(R &ar, R &ai, C a, C b) {
  ar = fma(a.x, b.x, ar);
  ar = fma(-a.y, b.y, ar);
  ai = fma(a.x, b.y, ai);
  ai = fma(a.y, b.x, ai);
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// ----------------------------------------------------------------------------- form

template <int D, typename R>
__global__ void __launch_bounds__(256) form_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const double *__restrict__ sigma,
                                                   const typename C2T<R>::T *__restrict__ Ff,
                                                   const typename C2T<R>::T *__restrict__ Fh,
                                                   typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                   int64_t slot_size, int Kmax) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  C *Z1 = reinterpret_cast<C *>(smem_raw);
  const Block blk = blocks[blockIdx.x];
  const int s = blockIdx.y;  // index along the half-range (last) axis
  const int K = blk.K, nl = 1 << blk.dl;
  const int64_t *lv = bleaves + blk.leaf0;
  C *out = phi + (int64_t)blk.slot * slot_size;

  if (D == 3) {
    C *Z2 = Z1 + (size_t)Kmax * Kmax;
    const int kk = k * k, k3 = kk * k;
    // Z1[J2][J1] = sum_J3 Fh3(s, J3) sigma(J3, J2, J1)
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
      const int J2 = idx / K, J1 = idx - J2 * K;
      const int o2 = J2 / k, j2 = J2 - o2 * k, o1 = J1 / k, j1 = J1 - o1 * k;
      R ar = 0, ai = 0;
      for (int o3 = 0; o3 < nl; ++o3) {
        const double *sp = sigma + lv[(o3 * nl + o2) * nl + o1] * k3 + j2 * k + j1;
        const C *fp = Fh + ((int64_t)(blk.mat[2] + o3) * nh + s) * k;
        for (int j3 = 0; j3 < k; ++j3) {
          const R v = (R)__ldg(sp + j3 * kk);
          const C f = fp[j3];
          ar = fma(f.x, v, ar);
          ai = fma(f.y, v, ai);
        }
      }
      Z1[idx] = C{ar, ai};
    }
    __syncthreads();
    // Z2[m2][J1] = sum_J2 Ff2(m2, J2) Z1[J2][J1]
    for (int idx = threadIdx.x; idx < n1 * K; idx += blockDim.x) {
      const int m2 = idx / K, J1 = idx - m2 * K;
      R ar = 0, ai = 0;
      for (int o2 = 0; o2 < nl; ++o2) {
        const C *fp = Ff + ((int64_t)(blk.mat[1] + o2) * n1 + m2) * k;
        const C *zp = Z1 + (o2 * k) * K + J1;
        for (int j2 = 0; j2 < k; ++j2) cfma(ar, ai, fp[j2], zp[j2 * K]);
      }
      Z2[idx] = C{ar, ai};
    }
    __syncthreads();
    // out[s][m2][m1] += sum_J1 Ff1(m1, J1) Z2[m2][J1]
    C *o = out + (int64_t)s * n1 * n1;
    for (int idx = threadIdx.x; idx < n1 * n1; idx += blockDim.x) {
      const int m2 = idx / n1, m1 = idx - m2 * n1;
      R ar = 0, ai = 0;
      for (int o1 = 0; o1 < nl; ++o1) {
        const C *fp = Ff + ((int64_t)(blk.mat[0] + o1) * n1 + m1) * k;
        const C *zp = Z2 + m2 * K + o1 * k;
        for (int j1 = 0; j1 < k; ++j1) cfma(ar, ai, fp[j1], zp[j1]);
      }
      atomicAdd(&o[idx].x, ar);
      atomicAdd(&o[idx].y, ai);
    }
  } else {
    const int kk = k * k;
    // Z1[J1] = sum_J2 Fh2(s, J2) sigma(J2, J1)
    for (int J1 = threadIdx.x; J1 < K; J1 += blockDim.x) {
      const int o1 = J1 / k, j1 = J1 - o1 * k;
      R ar = 0, ai = 0;
      for (int o2 = 0; o2 < nl; ++o2) {
        const double *sp = sigma + lv[o2 * nl + o1] * kk + j1;
        const C *fp = Fh + ((int64_t)(blk.mat[1] + o2) * nh + s) * k;
        for (int j2 = 0; j2 < k; ++j2) {
          const R v = (R)__ldg(sp + j2 * k);
          const C f = fp[j2];
          ar = fma(f.x, v, ar);
          ai = fma(f.y, v, ai);
        }
      }
      Z1[J1] = C{ar, ai};
    }
    __syncthreads();
    C *o = out + (int64_t)s * n1;
    for (int m1 = threadIdx.x; m1 < n1; m1 += blockDim.x) {
      R ar = 0, ai = 0;
      for (int o1 = 0; o1 < nl; ++o1) {
        const C *fp = Ff + ((int64_t)(blk.mat[0] + o1) * n1 + m1) * k;
        const C *zp = Z1 + o1 * k;
        for (int j1 = 0; j1 < k; ++j1) cfma(ar, ai, fp[j1], zp[j1]);
      }
      atomicAdd(&o[m1].x, ar);
      atomicAdd(&o[m1].y, ai);
    }
  }
}

// ----------------------------------------------------------------------------- evaluation

template <int D, typename R>
__global__ void __launch_bounds__(256) eval_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const typename C2T<R>::T *__restrict__ Ef,
                                                   const typename C2T<R>::T *__restrict__ Eh,
                                                   const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                   int k, int n1, int nh, int64_t slot_size) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  C *Y1 = reinterpret_cast<C *>(smem_raw);
  const Block blk = blocks[blockIdx.x];
  const int r = blockIdx.y;  // output index along the last axis
  if (r >= blk.K) return;
  const int K = blk.K, nl = 1 << blk.dl;
  const int64_t *lv = bleaves + blk.leaf0;
  const C *ps = psi + (int64_t)blk.slot * slot_size;
  const bool acc_u = (blk.flags & 1) != 0;
  const int od = r / k, td = r - od * k;
  const C *ed = Eh + ((int64_t)(blk.mat[D - 1] + od) * k + td) * nh;

  if (D == 3) {
    C *Y2 = Y1 + (size_t)n1 * n1;
    const int nn = n1 * n1, k3 = k * k * k;
    // Y1[m2][m1] = sum_m3 Eh3(r, m3) psi[m3][m2][m1]
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
      R ar = 0, ai = 0;
      for (int m3 = 0; m3 < nh; ++m3) cfma(ar, ai, ed[m3], ps[(int64_t)m3 * nn + idx]);
      Y1[idx] = C{ar, ai};
    }
    __syncthreads();
    // Y2[I2][m1] = sum_m2 Ef2(I2, m2) Y1[m2][m1]
    for (int idx = threadIdx.x; idx < K * n1; idx += blockDim.x) {
      const int I2 = idx / n1, m1 = idx - I2 * n1;
      const int o2 = I2 / k, t2 = I2 - o2 * k;
      const C *ep = Ef + ((int64_t)(blk.mat[1] + o2) * k + t2) * n1;
      R ar = 0, ai = 0;
      for (int m2 = 0; m2 < n1; ++m2) cfma(ar, ai, ep[m2], Y1[m2 * n1 + m1]);
      Y2[idx] = C{ar, ai};
    }
    __syncthreads();
    // u(r, I2, I1) = Re sum_m1 Ef1(I1, m1) Y2[I2][m1]
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
      const int I2 = idx / K, I1 = idx - I2 * K;
      const int o1 = I1 / k, t1 = I1 - o1 * k, o2 = I2 / k, t2 = I2 - o2 * k;
      const C *ep = Ef + ((int64_t)(blk.mat[0] + o1) * k + t1) * n1;
      const C *yp = Y2 + I2 * n1;
      R acc = 0;
      for (int m1 = 0; m1 < n1; ++m1) {
        const C e = ep[m1], y = yp[m1];
        acc = fma(e.x, y.x, acc);
        acc = fma(-e.y, y.y, acc);
      }
      double *up = u + lv[(od * nl + o2) * nl + o1] * k3 + (td * k + t2) * k + t1;
      if (acc_u) *up += (double)acc; else *up = (double)acc;
    }
  } else {
    const int kk = k * k;
    // Y1[m1] = sum_m2 Eh2(r, m2) psi[m2][m1]
    for (int m1 = threadIdx.x; m1 < n1; m1 += blockDim.x) {
      R ar = 0, ai = 0;
      for (int m2 = 0; m2 < nh; ++m2) cfma(ar, ai, ed[m2], ps[(int64_t)m2 * n1 + m1]);
      Y1[m1] = C{ar, ai};
    }
    __syncthreads();
    for (int I1 = threadIdx.x; I1 < K; I1 += blockDim.x) {
      const int o1 = I1 / k, t1 = I1 - o1 * k;
      const C *ep = Ef + ((int64_t)(blk.mat[0] + o1) * k + t1) * n1;
      R acc = 0;
      for (int m1 = 0; m1 < n1; ++m1) {
        const C e = ep[m1], y = Y1[m1];
        acc = fma(e.x, y.x, acc);
        acc = fma(-e.y, y.y, acc);
      }
      double *up = u + lv[od * nl + o1] * kk + td * k + t1;
      if (acc_u) *up += (double)acc; else *up = (double)acc;
    }
  }
}

// ----------------------------------------------------------------------------- diagonal shifts

template <int D>
__device__ __forceinline__ void mode_index(int64_t idx, int n1, int &m1, int &m2, int &m3) {
  m1 = (int)(idx % n1);
  const int64_t rest = idx / n1;
  if (D == 3) {
    m2 = (int)(rest % n1);
    m3 = (int)(rest / n1);
  } else {
    m2 = (int)rest;
    m3 = 0;
  }
}

// psi[dst] = sum_S T_out->in(S) phi[S].  The phase is a product of one 1D factor per axis,
// so the sum is taken axis by axis: sources arrive sorted by code (o_1 fastest), the x_1
// factor multiplies each source, the x_2 factor each run of equal (o_2, o_3), the x_3 factor
// each run of equal o_3 -- 27 + 9 + 3 complex products per mode in 3D instead of 27 x 3.
template <int D, typename R>
__global__ void gather_kernel(const int32_t *__restrict__ dst, const int64_t *__restrict__ ptr,
                              const GatherSrc *__restrict__ src, const typename C2T<R>::T *__restrict__ Pf,
                              const typename C2T<R>::T *__restrict__ Ph, const typename C2T<R>::T *__restrict__ phi,
                              typename C2T<R>::T *__restrict__ psi, int n1, int nh, int64_t slot_size) {
  using C = typename C2T<R>::T;
  const int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= slot_size) return;
  const int i = blockIdx.x;
  int m1, m2, m3;
  mode_index<D>(idx, n1, m1, m2, m3);
  // factors of the second and last axes (the last axis stores m >= 0 only)
  const C* P2 = (D == 3) ? Pf : Ph;
  const int s2 = (D == 3) ? n1 : nh, i2 = m2;
  R a1r = 0, a1i = 0, a2r = 0, a2i = 0, a3r = 0, a3i = 0;
  int g1 = -1, g2 = -1;  // current (o_2, o_3) run and o_3 run
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const GatherSrc g = src[q];
    const int run1 = g.code / 3, run2 = g.code / 9;
    if (run1 != g1) {
      if (g1 >= 0) {
        cfma(a2r, a2i, P2[(g1 % 3) * s2 + i2], C{a1r, a1i});
        a1r = a1i = 0;
      }
      g1 = run1;
    }
    if (D == 3 && run2 != g2) {
      if (g2 >= 0) {
        cfma(a3r, a3i, Ph[g2 * nh + m3], C{a2r, a2i});
        a2r = a2i = 0;
      }
      g2 = run2;
    }
    cfma(a1r, a1i, Pf[(g.code % 3) * n1 + m1], phi[(int64_t)g.slot * slot_size + idx]);
  }
  if (g1 >= 0) cfma(a2r, a2i, P2[(g1 % 3) * s2 + i2], C{a1r, a1i});
  if (D == 3) {
    if (g2 >= 0) cfma(a3r, a3i, Ph[g2 * nh + m3], C{a2r, a2i});
    psi[(int64_t)dst[i] * slot_size + idx] = C{a3r, a3i};
  } else {
    psi[(int64_t)dst[i] * slot_size + idx] = C{a2r, a2i};
  }
}

// phi[parent] = sum_children T_c->p(child) phi[child]
template <int D, typename R>
__global__ void merge_kernel(const TreeShift *__restrict__ items, const typename C2T<R>::T *__restrict__ qf,
                             const typename C2T<R>::T *__restrict__ qh, typename C2T<R>::T *__restrict__ phi, int n1,
                             int nh, int64_t slot_size) {
  using C = typename C2T<R>::T;
  const int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= slot_size) return;
  const TreeShift it = items[blockIdx.x];
  int m1, m2, m3;
  mode_index<D>(idx, n1, m1, m2, m3);
  R ar = 0, ai = 0;
  for (int c = 0; c < (1 << D); ++c) {
    const int b1 = c & 1, b2 = (c >> 1) & 1, b3 = (c >> 2) & 1;
    C ph = qf[b1 * n1 + m1];
    if (D == 3) {
      ph = cmul(ph, qf[b2 * n1 + m2]);
      ph = cmul(ph, qh[b3 * nh + m3]);
    } else {
      ph = cmul(ph, qh[b2 * nh + m2]);
    }
    cfma(ar, ai, ph, phi[(int64_t)it.child[c] * slot_size + idx]);
  }
  phi[(int64_t)it.parent * slot_size + idx] = C{ar, ai};
}

// psi[child] = T_p->c(child) psi[parent]
template <int D, typename R>
__global__ void push_kernel(const TreeShift *__restrict__ items, const typename C2T<R>::T *__restrict__ qf,
                            const typename C2T<R>::T *__restrict__ qh, typename C2T<R>::T *__restrict__ psi, int n1,
                            int nh, int64_t slot_size) {
  using C = typename C2T<R>::T;
  const int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= slot_size) return;
  const TreeShift it = items[blockIdx.x];
  int m1, m2, m3;
  mode_index<D>(idx, n1, m1, m2, m3);
  const C v = psi[(int64_t)it.parent * slot_size + idx];
  for (int c = 0; c < (1 << D); ++c) {
    const int b1 = c & 1, b2 = (c >> 1) & 1, b3 = (c >> 2) & 1;
    C ph = qf[b1 * n1 + m1];
    if (D == 3) {
      ph = cmul(ph, qf[b2 * n1 + m2]);
      ph = cmul(ph, qh[b3 * nh + m3]);
    } else {
      ph = cmul(ph, qh[b2 * nh + m2]);
    }
    psi[(int64_t)it.child[c] * slot_size + idx] = cmul(ph, v);
  }
}

// ----------------------------------------------------------------------------- near field

template <int D>
__global__ void __launch_bounds__(256) near_kernel(const int64_t *__restrict__ tgt, const int32_t *__restrict__ flags,
                                                   const int64_t *__restrict__ ptr, const NearSrc *__restrict__ src,
                                                   const double *__restrict__ tab, const double *__restrict__ sigma,
                                                   double *__restrict__ u, int k) {
  extern __shared__ double sm[];
  const int kk = k * k;
  const int np = (D == 3) ? kk * k : kk;
  double *s0 = sm, *A = sm + np, *B = A + np, *T = B + np;  // T: d tables of k x k
  constexpr int kMaxPer = (kMaxK * kMaxK * (D == 3 ? kMaxK : 1) + 255) / 256;
  double acc[kMaxPer];
#pragma unroll
  for (int q = 0; q < kMaxPer; ++q) acc[q] = 0.0;
  const int i = blockIdx.x;
  for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
    const NearSrc ns = src[p];
    const double *sg = sigma + ns.leaf * np;
    for (int e = threadIdx.x; e < np; e += blockDim.x) s0[e] = __ldg(sg + e);
    for (int e = threadIdx.x; e < D * kk; e += blockDim.x) {
      const int a = e / kk;
      T[e] = __ldg(tab + (int64_t)ns.tab[a] * kk + (e - a * kk));
    }
    __syncthreads();
    if (D == 3) {
      // A[j3][j2][t1] = sum_j1 T1[t1][j1] s0[j3][j2][j1]
      for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int row = e / k, t1 = e - row * k;
        const double *sp = s0 + row * k, *tp = T + t1 * k;
        double a = 0;
        for (int j = 0; j < k; ++j) a = fma(tp[j], sp[j], a);
        A[e] = a;
      }
      __syncthreads();
      // B[j3][t2][t1] = sum_j2 T2[t2][j2] A[j3][j2][t1]
      for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int j3 = e / kk, rem = e - j3 * kk, t2 = rem / k, t1 = rem - t2 * k;
        const double *tp = T + kk + t2 * k, *ap = A + j3 * kk + t1;
        double a = 0;
        for (int j = 0; j < k; ++j) a = fma(tp[j], ap[j * k], a);
        B[e] = a;
      }
      __syncthreads();
      // acc[t3][t2][t1] += sum_j3 T3[t3][j3] B[j3][t2][t1]
#pragma unroll
      for (int q = 0; q < kMaxPer; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < np) {
          const int t3 = e / kk, rem = e - t3 * kk;
          const double *tp = T + 2 * kk + t3 * k, *bp = B + rem;
          double a = acc[q];
          for (int j = 0; j < k; ++j) a = fma(tp[j], bp[j * kk], a);
          acc[q] = a;
        }
      }
    } else {
      // A[j2][t1] = sum_j1 T1[t1][j1] s0[j2][j1]
      for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int j2 = e / k, t1 = e - j2 * k;
        const double *sp = s0 + j2 * k, *tp = T + t1 * k;
        double a = 0;
        for (int j = 0; j < k; ++j) a = fma(tp[j], sp[j], a);
        A[e] = a;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kMaxPer; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < np) {
          const int t2 = e / k, t1 = e - t2 * k;
          const double *tp = T + kk + t2 * k, *ap = A + t1;
          double a = acc[q];
          for (int j = 0; j < k; ++j) a = fma(tp[j], ap[j * k], a);
          acc[q] = a;
        }
      }
    }
    __syncthreads();
  }
  double *ut = u + tgt[i] * np;
  const bool add = (flags[i] & 1) != 0;
#pragma unroll
  for (int q = 0; q < kMaxPer; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    if (e < np) {
      if (add) ut[e] += acc[q]; else ut[e] = acc[q];
    }
  }
}

// ----------------------------------------------------------------------------- host side

size_t form_smem_bytes(int d, int K, int n1, int prec) {
  const size_t c = prec ? sizeof(float2) : sizeof(double2);
  return d == 3 ? c * ((size_t)K * K + (size_t)n1 * K) : c * (size_t)K;
}

size_t eval_smem_bytes(int d, int K, int n1, int prec) {
  const size_t c = prec ? sizeof(float2) : sizeof(double2);
  return d == 3 ? c * ((size_t)n1 * n1 + (size_t)K * n1) : c * (size_t)n1;
}

int max_dynamic_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 48 * 1024;
  return v;
}

template <int D, typename R>
static cudaError_t run_typed(const ExecDesc &e, const double *sigma, double *u, cudaStream_t st) {
  using C = typename C2T<R>::T;
  cudaError_t err;
  C *phi = reinterpret_cast<C *>(e.phi);
  C *psi = reinterpret_cast<C *>(e.psi);
  const int n1 = e.n1, nh = e.nh;
  const int64_t ss = e.slot_size;
  const unsigned tiles = (unsigned)((ss + 255) / 256);

  auto mark = [&](int ph, int end) {
    if (e.events) cudaEventRecord(e.events[2 * ph + end], st);
  };
  mark(0, 0);
  if (e.n_blocks > 0) {
    // outgoing expansions: zero, then every block adds its contribution
    if ((err = cudaMemsetAsync(phi, 0, sizeof(C) * ss * e.n_phi_slots, st)) != cudaSuccess) return err;
    const size_t fsm = form_smem_bytes(D, e.Kmax, n1, sizeof(R) == 4);
    if ((err = cudaFuncSetAttribute(form_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm)) !=
        cudaSuccess)
      return err;
    form_kernel<D, R><<<dim3((unsigned)e.n_blocks, (unsigned)nh), 256, fsm, st>>>(
        e.blocks, e.block_leaves, sigma, reinterpret_cast<const C *>(e.Ff), reinterpret_cast<const C *>(e.Fh), phi,
        e.k, n1, nh, ss, e.Kmax);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  mark(0, 1);
  mark(1, 0);
  for (const ShiftStep &s : e.merge) {
    if (s.n == 0) continue;
    merge_kernel<D, R><<<dim3((unsigned)s.n, tiles), 256, 0, st>>>(
        s.items, reinterpret_cast<const C *>(s.qf), reinterpret_cast<const C *>(s.qh), phi, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  mark(1, 1);
  mark(2, 0);
  const C *eval_src = phi;
  if (!e.fourier && e.n_gather > 0) {
    gather_kernel<D, R><<<dim3((unsigned)e.n_gather, tiles), 256, 0, st>>>(
        e.gather_dst, e.gather_ptr, e.gather_src, reinterpret_cast<const C *>(e.Pf),
        reinterpret_cast<const C *>(e.Ph), phi, psi, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    eval_src = psi;
  }
  mark(2, 1);
  mark(3, 0);
  for (const ShiftStep &s : e.push) {
    if (s.n == 0) continue;
    push_kernel<D, R><<<dim3((unsigned)s.n, tiles), 256, 0, st>>>(
        s.items, reinterpret_cast<const C *>(s.qf), reinterpret_cast<const C *>(s.qh), psi, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  mark(3, 1);
  mark(4, 0);
  if (e.n_blocks > 0) {
    const size_t esm = eval_smem_bytes(D, e.Kmax, n1, sizeof(R) == 4);
    if ((err = cudaFuncSetAttribute(eval_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm)) !=
        cudaSuccess)
      return err;
    eval_kernel<D, R><<<dim3((unsigned)e.n_blocks, (unsigned)e.Kmax), 256, esm, st>>>(
        e.blocks, e.block_leaves, reinterpret_cast<const C *>(e.Ef), reinterpret_cast<const C *>(e.Eh), eval_src, u,
        e.k, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  mark(4, 1);
  mark(5, 0);
  if (e.n_near > 0) {
    const int np = D == 3 ? e.k * e.k * e.k : e.k * e.k;
    const size_t nsm = sizeof(double) * (3 * (size_t)np + (size_t)D * e.k * e.k);
    if ((err = cudaFuncSetAttribute(near_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm)) !=
        cudaSuccess)
      return err;
    near_kernel<D><<<(unsigned)e.n_near, 256, nsm, st>>>(e.near_tgt, e.near_flags, e.near_ptr, e.near_src, e.near_tab,
                                                         sigma, u, e.k);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  mark(5, 1);
  return cudaSuccess;
}

int launches_per_transform(const ExecDesc &e) {
  int n = 0;
  if (e.n_blocks > 0) n += 2;  // form + evaluate
  for (const ShiftStep &s : e.merge) n += s.n > 0;
  for (const ShiftStep &s : e.push) n += s.n > 0;
  if (!e.fourier && e.n_gather > 0) n += 1;
  if (e.n_near > 0) n += 1;
  return n;
}

cudaError_t run_transform(const ExecDesc &e, const double *sigma, double *u, cudaStream_t stream) {
  if (e.d == 3) return e.prec ? run_typed<3, float>(e, sigma, u, stream) : run_typed<3, double>(e, sigma, u, stream);
  return e.prec ? run_typed<2, float>(e, sigma, u, stream) : run_typed<2, double>(e, sigma, u, stream);
}

// ----------------------------------------------------------------------------- allocation-free variant
//
// For callers that cannot allocate device memory when they transform (for
// example code running under an allocator that forbids cudaMalloc, or a
// runtime that has already committed all device memory to its own pool), the
// expansion workspace can live in this fixed array instead of the plan's own.
// Every GPU that loads the library holds it until the process exits.  All
// calls share it: calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;
}  // namespace

cudaError_t noalloc_scratch(void **ptr) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    // host code only sees a stand-in for the array: ask the runtime for its device address
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_addr[dev] = p;
  }
  *ptr = g_scratch_addr[dev];
  return cudaSuccess;
}

cudaError_t run_transform_noalloc(const ExecDesc &e, const double *sigma, double *u, cudaStream_t stream) {
  void *base = nullptr;
  cudaError_t err = noalloc_scratch(&base);
  if (err != cudaSuccess) return err;
  const size_t c = e.prec ? sizeof(float2) : sizeof(double2);
  const size_t phi_bytes = c * (size_t)e.slot_size * (size_t)e.n_phi_slots;
  const size_t psi_bytes = c * (size_t)e.slot_size * (size_t)e.n_psi_slots;
  if (phi_bytes + psi_bytes > kNoallocScratchBytes) return cudaErrorInvalidValue;
  ExecDesc f = e;
  f.phi = base;
  f.psi = static_cast<unsigned char *>(base) + ((phi_bytes + 255) & ~(size_t)255);
  if (((phi_bytes + 255) & ~(size_t)255) + psi_bytes > kNoallocScratchBytes) return cudaErrorInvalidValue;
  f.events = nullptr;
  return run_transform(f, sigma, u, stream);
}

}  // namespace fgt
