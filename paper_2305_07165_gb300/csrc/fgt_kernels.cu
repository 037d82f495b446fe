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

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "fgt_exec.h"
#include "fgt_tables.h"
#include "fgt_tc.cuh"

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

// ----------------------------------------------------------------------------- checked build
//
// Built with -DFGT_CHECKED (libfgt_checked.so), every instrumented global access first checks that
// its bytes lie inside one of the buffers the host registered for the transform (sigma, u, the
// plan's tables and workspace).  A failing access is skipped, and the first failing site's source
// line is kept in g_check_word with a count in g_check_count, for the host to read: an
// out-of-range index becomes a reported error instead of a fault.  With no buffers registered
// (batched graphs), nothing is checked.  In the normal build FGT_OK_PTR is the constant true.
#ifdef FGT_CHECKED
struct CheckRanges {
  const char *lo[kCheckRanges];
  const char *hi[kCheckRanges];
  int n;
};
__device__ CheckRanges g_check_ranges;
__device__ unsigned int g_check_word, g_check_count;
__device__ __noinline__ bool chk_bytes(const void *p, size_t n, int site) {
  const CheckRanges &r = g_check_ranges;
  if (r.n == 0) return true;
  const char *c = static_cast<const char *>(p);
  for (int i = 0; i < r.n && i < kCheckRanges; ++i)
    if (c >= r.lo[i] && c + n <= r.hi[i]) return true;
  atomicCAS(&g_check_word, 0u, (unsigned)site);
  atomicAdd(&g_check_count, 1u);
  return false;
}
#define FGT_OK_PTR(p) ::fgt::chk_bytes((const void *)(p), sizeof(*(p)), __LINE__)
#define FGT_OK_BYTES(p, n) ::fgt::chk_bytes((const void *)(p), (size_t)(n), __LINE__)
#else
#define FGT_OK_PTR(p) true
#define FGT_OK_BYTES(p, n) true
#endif

// ----------------------------------------------------------------------------- form

template <int D, typename R>
__device__ __forceinline__ void form_body(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const double *__restrict__ sigma,
                                                   const typename C2T<R>::T *__restrict__ Ff,
                                                   const typename C2T<R>::T *__restrict__ Fh,
                                                   typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                   int64_t slot_size, int Kmax, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  C *Z1 = reinterpret_cast<C *>(smem_raw);
  const Block blk = blocks[bx];
  const int s = by;  // index along the half-range (last) axis
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
      if (FGT_OK_PTR(&o[idx])) {
        atomicAdd(&o[idx].x, ar);
        atomicAdd(&o[idx].y, ai);
      }
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
      if (FGT_OK_PTR(&o[m1])) {
        atomicAdd(&o[m1].x, ar);
        atomicAdd(&o[m1].y, ai);
      }
    }
  }
}


template <int D, typename R>
__global__ void __launch_bounds__(256) form_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const double *__restrict__ sigma,
                                                   const typename C2T<R>::T *__restrict__ Ff,
                                                   const typename C2T<R>::T *__restrict__ Fh,
                                                   typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                   int64_t slot_size, int Kmax) {
  form_body<D, R>(blocks, bleaves, sigma, Ff, Fh, phi, k, n1, nh, slot_size, Kmax, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- evaluation

template <int D, typename R>
__device__ __forceinline__ void eval_body(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const typename C2T<R>::T *__restrict__ Ef,
                                                   const typename C2T<R>::T *__restrict__ Eh,
                                                   const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                   int k, int n1, int nh, int64_t slot_size, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  C *Y1 = reinterpret_cast<C *>(smem_raw);
  const Block blk = blocks[bx];
  const int r = by;  // output index along the last axis
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
      if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc); else *up = (double)acc; }
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
      if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc); else *up = (double)acc; }
    }
  }
}


template <int D, typename R>
__global__ void __launch_bounds__(256) eval_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                   const typename C2T<R>::T *__restrict__ Ef,
                                                   const typename C2T<R>::T *__restrict__ Eh,
                                                   const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                   int k, int n1, int nh, int64_t slot_size) {
  eval_body<D, R>(blocks, bleaves, Ef, Eh, psi, u, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- grouped form

// A CTA takes up to G blocks of one anchor (same K) and one m_d plane: their sigma (converted
// to R) and 1D matrices are staged in shared memory, the three contractions run for all its
// blocks, and their summed contribution goes to the anchor slot with one atomic per
// coefficient (G times fewer atomics than one CTA per block).  The x_1 matrices are stored transposed ([J][m]) so that
// threads reading consecutive modes hit consecutive banks.
template <int D, typename R>
__device__ __forceinline__ void form2_body(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma,
                                                    const typename C2T<R>::T *__restrict__ Ff,
                                                    const typename C2T<R>::T *__restrict__ Fh,
                                                    typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  const int b0 = gptr[bx], G = gptr[bx + 1] - b0;
  const Block B0 = blocks[b0];
  const int K = B0.K, nl = 1 << B0.dl;
  const int KK = K * K, npb = (D == 3) ? KK * K : KK, kp = (D == 3) ? k * k * k : k * k;
  // layout
  R *sig = reinterpret_cast<R *>(smem_raw);
  const size_t sig_bytes = ((size_t)G * npb * sizeof(R) + 15) & ~(size_t)15;  // keep C aligned
  C *F1t = reinterpret_cast<C *>(smem_raw + sig_bytes);         // [G][K][n1]
  C *Fd = F1t + (size_t)G * K * n1;                             // [G][nh][K]
  C *Z1 = Fd + (size_t)G * nh * K;                              // [G][K^(D-1)]
  C *F2 = Z1 + (size_t)G * (D == 3 ? KK : K);                   // [G][n1][K]   (3D)
  C *Z2 = F2 + (size_t)G * n1 * K;                              // [G][n1][K]   (3D)
  for (int g = 0; g < G; ++g) {
    const Block b = blocks[b0 + g];
    const int64_t *lv = bleaves + b.leaf0;
    for (int e = threadIdx.x; e < npb; e += blockDim.x) {
      int J1 = e % K, rest = e / K, J2 = (D == 3) ? rest % K : rest, J3 = (D == 3) ? rest / K : 0;
      const int o1 = J1 / k, o2 = J2 / k, o3 = J3 / k;
      const int64_t leaf = (D == 3) ? lv[(o3 * nl + o2) * nl + o1] : lv[o2 * nl + o1];
      const int node = (D == 3) ? ((J3 - o3 * k) * k + (J2 - o2 * k)) * k + (J1 - o1 * k) : (J2 - o2 * k) * k + (J1 - o1 * k);
      sig[(size_t)g * npb + e] = (R)__ldg(sigma + leaf * kp + node);
    }
    for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
      const int J = e / n1, m = e - J * n1;
      F1t[(size_t)g * K * n1 + e] = Ff[((int64_t)(b.mat[0] + J / k) * n1 + m) * k + J % k];
    }
    for (int e = threadIdx.x; e < nh * K; e += blockDim.x) {
      const int m = e / K, J = e - m * K;
      Fd[(size_t)g * nh * K + e] = Fh[((int64_t)(b.mat[D - 1] + J / k) * nh + m) * k + J % k];
    }
    if (D == 3)
      for (int e = threadIdx.x; e < n1 * K; e += blockDim.x) {
        const int m = e / K, J = e - m * K;
        F2[(size_t)g * n1 * K + e] = Ff[((int64_t)(b.mat[1] + J / k) * n1 + m) * k + J % k];
      }
  }
  __syncthreads();
  C *out = phi + (int64_t)B0.slot * slot_size;
  {
    const int s = by;  // one m_d plane per CTA
    if (D == 3) {
      // Z1[g][J2][J1] = sum_J3 Fd[g][s][J3] sig[g][J3][J2][J1]
      for (int e = threadIdx.x; e < G * KK; e += blockDim.x) {
        const int g = e / KK, rem = e - g * KK;
        const R *sp = sig + (size_t)g * npb + rem;
        const C *fp = Fd + ((size_t)g * nh + s) * K;
        R ar = 0, ai = 0;
        for (int J3 = 0; J3 < K; ++J3) {
          const R v = sp[(size_t)J3 * KK];
          const C f = fp[J3];
          ar = fma(f.x, v, ar);
          ai = fma(f.y, v, ai);
        }
        Z1[e] = C{ar, ai};
      }
      __syncthreads();
      // Z2[g][m2][J1] = sum_J2 F2[g][m2][J2] Z1[g][J2][J1]
      for (int e = threadIdx.x; e < G * n1 * K; e += blockDim.x) {
        const int g = e / (n1 * K), rem = e - g * n1 * K, m2 = rem / K, J1 = rem - m2 * K;
        const C *fp = F2 + ((size_t)g * n1 + m2) * K;
        const C *zp = Z1 + (size_t)g * KK + J1;
        R ar = 0, ai = 0;
        for (int J2 = 0; J2 < K; ++J2) cfma(ar, ai, fp[J2], zp[J2 * K]);
        Z2[e] = C{ar, ai};
      }
      __syncthreads();
      // out[s][m2][m1] += sum_g sum_J1 F1[g][m1][J1] Z2[g][m2][J1]
      C *o = out + (int64_t)s * n1 * n1;
      for (int idx = threadIdx.x; idx < n1 * n1; idx += blockDim.x) {
        const int m2 = idx / n1, m1 = idx - m2 * n1;
        R ar = 0, ai = 0;
        for (int g = 0; g < G; ++g) {
          const C *fp = F1t + (size_t)g * K * n1 + m1;
          const C *zp = Z2 + ((size_t)g * n1 + m2) * K;
          for (int J1 = 0; J1 < K; ++J1) cfma(ar, ai, fp[J1 * n1], zp[J1]);
        }
        if (FGT_OK_PTR(&o[idx])) {
          atomicAdd(&o[idx].x, ar);
          atomicAdd(&o[idx].y, ai);
        }
      }
      __syncthreads();
    } else {
      // Z1[g][J1] = sum_J2 Fd[g][s][J2] sig[g][J2][J1]
      for (int e = threadIdx.x; e < G * K; e += blockDim.x) {
        const int g = e / K, J1 = e - g * K;
        const R *sp = sig + (size_t)g * npb + J1;
        const C *fp = Fd + ((size_t)g * nh + s) * K;
        R ar = 0, ai = 0;
        for (int J2 = 0; J2 < K; ++J2) {
          const R v = sp[(size_t)J2 * K];
          const C f = fp[J2];
          ar = fma(f.x, v, ar);
          ai = fma(f.y, v, ai);
        }
        Z1[e] = C{ar, ai};
      }
      __syncthreads();
      C *o = out + (int64_t)s * n1;
      for (int m1 = threadIdx.x; m1 < n1; m1 += blockDim.x) {
        R ar = 0, ai = 0;
        for (int g = 0; g < G; ++g) {
          const C *fp = F1t + (size_t)g * K * n1 + m1;
          const C *zp = Z1 + (size_t)g * K;
          for (int J1 = 0; J1 < K; ++J1) cfma(ar, ai, fp[J1 * n1], zp[J1]);
        }
        if (FGT_OK_PTR(&o[m1])) {
          atomicAdd(&o[m1].x, ar);
          atomicAdd(&o[m1].y, ai);
        }
      }
      __syncthreads();
    }
  }
}


template <int D, typename R>
__global__ void __launch_bounds__(256) form2_kernel(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma,
                                                    const typename C2T<R>::T *__restrict__ Ff,
                                                    const typename C2T<R>::T *__restrict__ Fh,
                                                    typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size) {
  form2_body<D, R>(blocks, gptr, bleaves, sigma, Ff, Fh, phi, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- register-tiled form (3D)
//
// A CTA takes a group of G blocks of one anchor (same K) and a chunk of up to kSc planes m_3.
// Stage 1 (J3 -> m3) keeps kSc outputs per thread, stages 2 (J2 -> m2) and 3 (J1 -> m1) run as
// small complex GEMMs with 4 x 4 register tiles, so every operand read from shared memory
// feeds four complex multiply-adds.  The group's contributions are summed before one atomic
// add per coefficient.
constexpr int kSc = 4;

__host__ __device__ inline int pad_gk(int GK) { return GK + 1; }  // row stride of Z2 (bank spread)

// ----------------------------------------------------------------------------- FP64 tensor-core tiles
//
// FP64 on the tensor cores: mma.m8n8k4 with f64 operands and accumulators (exact FP64 products,
// only the summation order differs from the CUDA-core kernels).  A complex product C = A B is
// embedded in real ones over an interleaved (re, im) contraction index (see the 3xTF32 helpers
// below for the same embedding).  Fragments, g = lane / 4, t = lane % 4: a = A[g][t],
// b = B[t][g], c = {C[g][2t], C[g][2t+1]}.
__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// One warp: rows i0 .. i0+7 of C (+)= A B for NBLK blocks of 8 columns from j0, A [arows][kc]
// (row stride lda), B [kc][ncols] (row stride ldb), complex FP64.  acc[2 b] holds the real parts
// of column block b, acc[2 b + 1] the imaginary parts.
template <int NBLK>
__device__ __forceinline__ void zgemm8_dmma(double (&acc)[2 * NBLK][2], const double2 *A, int lda, int arows, int i0,
                                            const double2 *B, int ldb, int ncols, int j0, int kc) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int row = i0 + g;
  for (int k0 = 0; k0 < 2 * kc; k0 += 4) {
    const int kr = k0 + t, J = kr >> 1, part = kr & 1;
    const bool kin = J < kc;
    double a = 0.0;
    if (kin && row < arows) {
      const double2 v = A[(size_t)row * lda + J];
      a = part ? v.y : v.x;
    }
#pragma unroll
    for (int b = 0; b < NBLK; ++b) {
      const int col = j0 + b * 8 + g;
      double2 f = make_double2(0.0, 0.0);
      if (kin && col < ncols) f = B[(size_t)J * ldb + col];
      dmma(acc[2 * b], a, part ? -f.y : f.x);
      dmma(acc[2 * b + 1], a, part ? f.x : f.y);
    }
  }
}

template <typename R, bool TC>  // TC (FP64 only): stage 3 on the tensor cores (DMMA)
__device__ __forceinline__ void form3_body(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma,
                                                    const typename C2T<R>::T *__restrict__ Ff,
                                                    const typename C2T<R>::T *__restrict__ Fh,
                                                    typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  const int b0 = gptr[bx], G = gptr[bx + 1] - b0;
  const Block B0 = blocks[b0];
  const int K = B0.K, nl = 1 << B0.dl;
  const int KK = K * K, npb = KK * K, kp = k * k * k, GK = G * K, ldz = pad_gk(GK);
  const int s0 = by * kSc, ns = min(kSc, nh - s0);
  R *sig = reinterpret_cast<R *>(smem_raw);                                   // [G][K^3]
  const size_t sig_bytes = ((size_t)G * npb * sizeof(R) + 15) & ~(size_t)15;
  C *F1t = reinterpret_cast<C *>(smem_raw + sig_bytes);                       // [G K][n1]
  C *F2 = F1t + (size_t)GK * n1;                                              // [G][n1][K]
  C *Fd = F2 + (size_t)G * n1 * K;                                            // [G][kSc][K]
  C *Z1 = Fd + (size_t)G * kSc * K;                                           // [kSc][G][K][K]
  C *Z2 = Z1 + (size_t)kSc * G * KK;                                          // [kSc][n1][ldz]
  for (int g = 0; g < G; ++g) {
    const Block b = blocks[b0 + g];
    const int64_t *lv = bleaves + b.leaf0;
    // sigma of the block, leaf by leaf (k^3 contiguous values per leaf)
    for (int e = threadIdx.x; e < npb; e += blockDim.x) {
      const int leafi = e / kp, node = e - leafi * kp;
      const int o1 = leafi % nl, o2 = (leafi / nl) % nl, o3 = leafi / (nl * nl);
      const int j1 = node % k, j2 = (node / k) % k, j3 = node / (k * k);
      sig[(size_t)g * npb + ((o3 * k + j3) * K + (o2 * k + j2)) * K + (o1 * k + j1)] =
          (R)__ldg(sigma + lv[leafi] * kp + node);
    }
    for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
      const int J = e / n1, m = e - J * n1;
      F1t[(size_t)(g * K + J) * n1 + m] = Ff[((int64_t)(b.mat[0] + J / k) * n1 + m) * k + J % k];
    }
    for (int e = threadIdx.x; e < n1 * K; e += blockDim.x) {
      const int m = e / K, J = e - m * K;
      F2[(size_t)g * n1 * K + e] = Ff[((int64_t)(b.mat[1] + J / k) * n1 + m) * k + J % k];
    }
    for (int e = threadIdx.x; e < kSc * K; e += blockDim.x) {
      const int q = e / K, J = e - q * K;
      Fd[((size_t)g * kSc + q) * K + J] =
          (q < ns) ? Fh[((int64_t)(b.mat[2] + J / k) * nh + s0 + q) * k + J % k] : C{0, 0};
    }
  }
  __syncthreads();
  // stage 1: Z1[q][g][J2][J1] = sum_J3 Fd[g][q][J3] sig[g][J3][J2][J1], all kSc planes per thread
  for (int e = threadIdx.x; e < G * KK; e += blockDim.x) {
    const int g = e / KK, rem = e - g * KK;
    const R *sp = sig + (size_t)g * npb + rem;
    const C *fp = Fd + (size_t)g * kSc * K;
    R ar[kSc], ai[kSc];
#pragma unroll
    for (int q = 0; q < kSc; ++q) ar[q] = ai[q] = 0;
    for (int J3 = 0; J3 < K; ++J3) {
      const R v = sp[(size_t)J3 * KK];
#pragma unroll
      for (int q = 0; q < kSc; ++q) {
        const C f = fp[q * K + J3];
        ar[q] = fma(f.x, v, ar[q]);
        ai[q] = fma(f.y, v, ai[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kSc; ++q) Z1[((size_t)q * G + g) * KK + rem] = C{ar[q], ai[q]};
  }
  __syncthreads();
  // stage 2: Z2[q][m2][g K + J1] = sum_J2 F2[g][m2][J2] Z1[q][g][J2][J1]; 4 x 4 tiles over (m2, J1)
  {
    const int tm = (n1 + 3) / 4, tj = (K + 3) / 4, ntile = ns * G * tm * tj;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      int r = t;
      const int bj = r % tj; r /= tj;
      const int bm = r % tm; r /= tm;
      const int g = r % G, q = r / G;
      R ar[4][4], ai[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0;
      const C *fp = F2 + (size_t)g * n1 * K;
      const C *zp = Z1 + ((size_t)q * G + g) * KK;
      for (int J2 = 0; J2 < K; ++J2) {
        C a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = bm * 4 + i;
          a[i] = (m < n1) ? fp[m * K + J2] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int J1 = bj * 4 + j;
          b[j] = (J1 < K) ? zp[J2 * K + J1] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(ar[i][j], ai[i][j], a[i], b[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m = bm * 4 + i, J1 = bj * 4 + j;
          if (m < n1 && J1 < K) Z2[((size_t)q * n1 + m) * ldz + g * K + J1] = C{ar[i][j], ai[i][j]};
        }
    }
  }
  __syncthreads();
  // stage 3: out[s0+q][m2][m1] += sum_{gJ} Z2[q][m2][gJ] F1t[gJ][m1]; 4 x 4 tiles over (m2, m1)
  C *out = phi + (int64_t)B0.slot * slot_size;
  if constexpr (TC && sizeof(R) == 8) {
    // one warp per (plane, 8 rows of m2, 32 columns of m1)
    const int mt = (n1 + 7) / 8, cb = (n1 + 31) / 32;
    for (int job = threadIdx.x >> 5; job < ns * mt * cb; job += blockDim.x >> 5) {
      const int c0 = job % cb, rest = job / cb, bm = rest % mt, q = rest / mt;
      double acc[8][2];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = 0.0;
      zgemm8_dmma<4>(acc, Z2 + (size_t)q * n1 * ldz, ldz, n1, bm * 8, F1t, n1, n1, c0 * 32, GK);
      const int lane = threadIdx.x & 31, m2 = bm * 8 + (lane >> 2);
      C *o = out + (int64_t)(s0 + q) * n1 * n1;
      if (m2 < n1) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int m1 = c0 * 32 + b * 8 + 2 * (lane & 3) + c;
            if (m1 < n1) {
              if (FGT_OK_PTR(&o[m2 * n1 + m1])) {
                atomicAdd(&o[m2 * n1 + m1].x, acc[2 * b][c]);
                atomicAdd(&o[m2 * n1 + m1].y, acc[2 * b + 1][c]);
              }
            }
          }
      }
    }
  } else {
    const int tm = (n1 + 3) / 4, ntile = ns * tm * tm;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const int b1 = t % tm, rest = t / tm, b2 = rest % tm, q = rest / tm;
      R ar[4][4], ai[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0;
      const C *zq = Z2 + (size_t)q * n1 * ldz;
      for (int J = 0; J < GK; ++J) {
        C a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m2 = b2 * 4 + i;
          a[i] = (m2 < n1) ? zq[(size_t)m2 * ldz + J] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m1 = b1 * 4 + j;
          b[j] = (m1 < n1) ? F1t[(size_t)J * n1 + m1] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(ar[i][j], ai[i][j], a[i], b[j]);
      }
      C *o = out + (int64_t)(s0 + q) * n1 * n1;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m2 = b2 * 4 + i, m1 = b1 * 4 + j;
          if (m2 < n1 && m1 < n1) {
            if (FGT_OK_PTR(&o[m2 * n1 + m1])) {
              atomicAdd(&o[m2 * n1 + m1].x, ar[i][j]);
              atomicAdd(&o[m2 * n1 + m1].y, ai[i][j]);
            }
          }
        }
    }
  }
}


template <typename R, bool TC>  // TC (FP64 only): stage 3 on the tensor cores (DMMA)
__global__ void __launch_bounds__(256) form3_kernel(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma,
                                                    const typename C2T<R>::T *__restrict__ Ff,
                                                    const typename C2T<R>::T *__restrict__ Fh,
                                                    typename C2T<R>::T *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size) {
  form3_body<R, TC>(blocks, gptr, bleaves, sigma, Ff, Fh, phi, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- 3xTF32 tensor-core helpers
//
// Split-precision contractions on the tensor cores: every FP32 operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a product is accumulated as
// a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32 (the a_lo b_lo term is below FP32 rounding).
// A complex product C = A B is embedded in one real product over an interleaved (re, im)
// contraction index: C_re = sum_k A~[k] Bre~[k], C_im = sum_k A~[k] Bim~[k] with
// A~[2j] = Re A_j, A~[2j+1] = Im A_j, Bre~[2j] = Re B_j, Bre~[2j+1] = -Im B_j,
// Bim~[2j] = Im B_j, Bim~[2j+1] = Re B_j.
// Fragments of mma.m16n8k8 (TF32, A row-major, B column-major), g = lane / 4, t = lane % 4:
// a = {A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4]}, b = {B[t][g], B[t+4][g]},
// c = {C[g][2t], C[g][2t+1], C[g+8][2t], C[g+8][2t+1]}.

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += a b in 3xTF32 (small terms first)
__device__ __forceinline__ void mma3(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                     uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  mma_tf32(c, al, bh0, bh1);
  mma_tf32(c, ah, bl0, bl1);
  mma_tf32(c, ah, bh0, bh1);
}

// ----------------------------------------------------------------------------- packed FP32 sigma (3D)
//
// One CTA per block_leaves entry: the leaf's k^3 values, converted to FP32, go to their place in
// the block's (J3, J2, J1) tile at sigp + block.leaf0 k^3, so that every form CTA that needs
// the block reads it as one contiguous run.
// FP64 <-> FP32 conversions on the integer pipes.  GB300 executes F2F conversions involving FP64 on
// its narrow FP64 pipe (2 results per clock per SM); these take a dozen integer operations instead.
// Round to nearest even, as the hardware conversion; magnitudes below FP32's normal range (2^-126,
// far below any value that matters next to |u|) become a signed zero; overflow gives infinity.
__device__ __forceinline__ float f64_to_f32_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b, s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(s);
  if (e >= 255) return __uint_as_float(s | 0x7F800000u);
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29), rest = lo & 0x1FFFFFFFu;
  uint32_t r = s | ((uint32_t)e << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;  // a carry moves into the exponent
  return __uint_as_float(r);
}
__device__ __forceinline__ double f32_to_f64_int(uint32_t b) {
  const uint32_t s = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e == 0) return __hiloint2double((int)s, 0);                 // zero; subnormals flushed
  if (e == 255) return __hiloint2double((int)(s | 0x7FF00000u | (m >> 3)), (int)(m << 29));  // inf / nan
  return __hiloint2double((int)(s | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// ---- double-float arithmetic: a value as the unevaluated sum hi + lo of two FP32 numbers (about
// 48 significant bits), on GB300's FP32 pipes (64 times the FP64 rate).  The error-free sum of
// Knuth and the FMA product error (the exact a*b - RN(a*b)) give a fused multiply-add whose error
// is about 2^-47 of its terms; conversions to and from FP64 use integer operations only.
struct dfl {
  float hi, lo;
};

// x rounded to 24 bits (hi) and the rest (lo, rounded to 24 bits: |lo| <= 2^-24 |hi|); zero when
// |x| < 2^-126 (subnormal FP32 range), lo zero when it would be.
__device__ __forceinline__ dfl dfl_from_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e - 896 <= 0 || e - 896 >= 255) return dfl{0.f, 0.f};
  const unsigned s = (unsigned)(b >> 63) << 31;
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));  // x = m 2^(e - 1075)
  const long long mh = (m + (1LL << 28)) >> 29;                              // 24 bits, or 2^24 on a carry
  const int r = (int)(m - (mh << 29));                                       // |r| <= 2^28
  // mh - 2^23 is the mantissa field; a carry (mh = 2^24) moves into the exponent
  const float h = __uint_as_float((s | ((unsigned)(e - 896) << 23)) + (unsigned)(mh - (1LL << 23)));
  float lo = 0.f;
  if (e - 948 >= 1 && r != 0) {
    const float sc = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
    lo = (float)r * sc;
    if (s) lo = -lo;
  }
  return dfl{h, lo};
}

// hi + lo rounded to FP64 (integer operations).
__device__ __forceinline__ double dfl_to_f64(dfl a) {
  const uint32_t bh = __float_as_uint(a.hi), bl = __float_as_uint(a.lo);
  const int eh = (int)((bh >> 23) & 0xFF), el = (int)((bl >> 23) & 0xFF);
  if (eh == 0) return f32_to_f64_int(bl);
  long long Mh = (long long)((bh & 0x7FFFFF) | 0x800000);
  if (bh >> 31) Mh = -Mh;
  long long V = Mh << 29;  // value = V 2^(eh - 150 - 29)
  if (el != 0) {
    long long Ml = (long long)((bl & 0x7FFFFF) | 0x800000);
    if (bl >> 31) Ml = -Ml;
    const int d = eh - el;  // lo's units below hi's
    if (d <= 29) V += Ml << (29 - d);
    else if (d < 29 + 26) V += (Ml + (1LL << (d - 30))) >> (d - 29);
  }
  return i64_to_f64_scaled(V, eh - 150 - 29);
}

// a + b in double-float
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  const float sm = a.hi + b.hi, bb = sm - a.hi;
  float t = (a.hi - (sm - bb)) + (b.hi - bb);
  t += a.lo + b.lo;
  const float hi = sm + t;
  return dfl{hi, t - (hi - sm)};
}
__device__ __forceinline__ dfl dfl_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

// a b + c in double-float
__device__ __forceinline__ dfl dfl_fma(dfl a, dfl b, dfl c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float sm = p + c.hi, bb = sm - p;
  float t = (p - (sm - bb)) + (c.hi - bb);
  t += e + c.lo;
  const float hi = sm + t;
  return dfl{hi, t - (hi - sm)};
}

__device__ __forceinline__ void sigma_pack_body(const Block *__restrict__ blocks,
                                                         const int32_t *__restrict__ pack_block,
                                                         const int64_t *__restrict__ bleaves,
                                                         const double *__restrict__ sigma, float *__restrict__ sigp,
                                                         int k, int bx, int by) {
  const int64_t i = bx;
  const Block b = blocks[pack_block[i]];
  const bool j3_fastest = (b.flags & 4) != 0;  // the block is formed by the tcgen05 form
  const int kp = k * k * k, nl = 1 << b.dl, K = b.K;
  const int leafi = (int)(i - b.leaf0);
  const int o1 = leafi % nl, o2 = (leafi / nl) % nl, o3 = leafi / (nl * nl);
  const double *src = sigma + bleaves[i] * kp;
  float *dst = sigp + b.leaf0 * kp;
  __shared__ float leaf[kMaxK * kMaxK * kMaxK];  // the leaf's values, node index j1 fastest
  if (k == 8) {
    // k = 8 (K = nl 8, a power of two): shifts, and the staging rows padded to 65 floats per j3 plane
    // so that reading along j3 (stride 65) or along j1 (stride 1) is free of bank conflicts
    for (int n2 = threadIdx.x; n2 < 256; n2 += blockDim.x) {
      const int node = 2 * n2;
      double2 v = make_double2(0.0, 0.0);
      if (FGT_OK_BYTES(src + node, 16)) v = __ldg(reinterpret_cast<const double2 *>(src + node));
      const int j3 = node >> 6, r = node & 63;
      // one value through the FP64 pipe's conversion, one through the integer pipes: the two run
      // side by side (all on the integer pipes, the pack was issue-bound; all on the FP64 pipe, that
      // narrow pipe would be the limit)
      leaf[j3 * 65 + r] = __double2float_rn(v.x);
      leaf[j3 * 65 + r + 1] = f64_to_f32_int(v.y);
    }
    __syncthreads();
    const int lK = __ffs(K) - 1;
    for (int t = threadIdx.x; t < 512; t += blockDim.x) {
      const int a = t & 7, bq = (t >> 3) & 7, c = t >> 6;  // fastest, middle, slowest index of the run order
      float *dp;
      float v;
      if (j3_fastest) {  // a = j3, bq = j2, c = j1
        dp = dst + (((((o1 << 3) + c) << lK) + (o2 << 3) + bq) << lK) + (o3 << 3) + a;
        v = leaf[a * 65 + (bq << 3) + c];
      } else {           // a = j1, bq = j2, c = j3
        dp = dst + (((((o3 << 3) + c) << lK) + (o2 << 3) + bq) << lK) + (o1 << 3) + a;
        v = leaf[c * 65 + (bq << 3) + a];
      }
      if (FGT_OK_PTR(dp)) *dp = v;
    }
    return;
  }
  for (int node = threadIdx.x; node < kp; node += blockDim.x)
    if (FGT_OK_PTR(src + node)) leaf[node] = f64_to_f32_int(__ldg(src + node));
  __syncthreads();
  // written in runs of k consecutive floats: (J3, J2, J1) order for the CUDA-core forms (J1
  // fastest), (J1, J2, J3) for the tcgen05 form (J3 fastest)
  for (int t = threadIdx.x; t < kp; t += blockDim.x) {
    const int a = t % k, bq = (t / k) % k, c = t / (k * k);  // fastest, middle, slowest index of the run order
    float *dp;
    float v;
    if (j3_fastest) {  // a = j3, bq = j2, c = j1
      dp = dst + ((o1 * k + c) * K + (o2 * k + bq)) * K + (o3 * k + a);
      v = leaf[(a * k + bq) * k + c];
    } else {           // a = j1, bq = j2, c = j3
      dp = dst + ((o3 * k + c) * K + (o2 * k + bq)) * K + (o1 * k + a);
      v = leaf[t];
    }
    if (FGT_OK_PTR(dp)) *dp = v;
  }
}


__global__ void __launch_bounds__(256) sigma_pack_kernel(const Block *__restrict__ blocks,
                                                         const int32_t *__restrict__ pack_block,
                                                         const int64_t *__restrict__ bleaves,
                                                         const double *__restrict__ sigma, float *__restrict__ sigp,
                                                         int k) {
  sigma_pack_body(blocks, pack_block, bleaves, sigma, sigp, k, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- tensor-core form (3D, FP32)
//
// Same work split as form3_kernel; stages 1-2 on the CUDA cores, stage 3 (the largest,
// Z2 (n1 x GK) times F1 (GK x n1) per plane) on the tensor cores in 3xTF32.  F1 is embedded
// once per CTA into split B operands Bh / Bl of 2*n1p columns (re outputs, then im outputs)
// by 2*GK interleaved rows.
constexpr int kNbtMax = 14;  // n-tiles of 8 columns: 2 * n1p / 8 <= 14 (n1 <= 56)

__host__ __device__ inline int n1_pad8(int n1) { return (n1 + 7) / 8 * 8; }
__host__ __device__ inline int ldz4(int GK) { return GK + 2; }       // complex row stride of Z2
__host__ __device__ inline int ldb4(int GK) { return 2 * GK + 4; }   // uint32 row stride of Bh / Bl

template <int NBT, bool BIG>  // NBT: n-tiles of 8 output columns held in registers (>= 2 n1p / 8)
__device__ __forceinline__ void form4_body(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma, const float *__restrict__ sigp,
                                                    const float2 *__restrict__ Ff, const float2 *__restrict__ Fh,
                                                    float2 *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size, int bx, int by) {
  using R = float;
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem4[];
  // linear grid, plane chunk fastest: the CTAs of one group run close together and share its
  // sigma and matrices in L2
  const int nchunk = (nh + kSc - 1) / kSc;
  const int grp = (int)(bx / nchunk), chunk = (int)(bx - (unsigned)grp * nchunk);
  const int b0 = gptr[grp], G = gptr[grp + 1] - b0;
  const Block B0 = blocks[b0];
  const int K = B0.K, nl = 1 << B0.dl;
  const int KK = K * K, npb = KK * K, kp = k * k * k, GK = G * K, ldz = ldz4(GK), ldb = ldb4(GK);
  const int n1p = n1_pad8(n1), NB = 2 * n1p;
  const int s0 = chunk * kSc, ns = min(kSc, nh - s0);
  // F1t and Z2 live through stage 3; sigma, F2, Fd and Z1 are dead after stage 2, and the split
  // B operands of stage 3 are built over them.  BIG (one block of K > 16): no sigma tile,
  // stage 1 streams it from global memory.
  C *F1t = reinterpret_cast<C *>(smem4);                                      // [G K][n1]
  C *Z2 = F1t + (size_t)GK * n1;                                              // [kSc][n1][ldz]
  unsigned char *s12 = reinterpret_cast<unsigned char *>(Z2 + (size_t)kSc * n1 * ldz);
  R *sig = reinterpret_cast<R *>(s12);                                        // [G][K^3]
  const size_t sig_bytes = BIG ? 0 : ((size_t)G * npb * sizeof(R) + 15) & ~(size_t)15;
  C *F2 = reinterpret_cast<C *>(s12 + sig_bytes);                             // [G][n1][K]
  C *Fd = F2 + (size_t)G * n1 * K;                                            // [G][kSc][K]
  C *Z1 = Fd + (size_t)G * kSc * K;                                           // [kSc][G][K][K]
  uint32_t *Bh = reinterpret_cast<uint32_t *>(s12);                           // [NB][ldb], after stage 2
  uint32_t *Bl = Bh + (size_t)NB * ldb;
  for (int g = 0; g < G; ++g) {
    const Block b = blocks[b0 + g];
    if (!BIG) {
      if (sigp != nullptr) {
        // packed FP32 sigma: the block's K^3 values are contiguous and already in tile order
        const float *src = sigp + b.leaf0 * kp;
        if ((kp & 3) == 0) {
          const float4 *s4 = reinterpret_cast<const float4 *>(src);
          float4 *d4 = reinterpret_cast<float4 *>(sig + (size_t)g * npb);
          for (int e = threadIdx.x; e < (npb >> 2); e += blockDim.x) d4[e] = __ldg(s4 + e);
        } else {
          for (int e = threadIdx.x; e < npb; e += blockDim.x) sig[(size_t)g * npb + e] = __ldg(src + e);
        }
      } else {
        const int64_t *lv = bleaves + b.leaf0;
        for (int e = threadIdx.x; e < npb; e += blockDim.x) {
          const int leafi = e / kp, node = e - leafi * kp;
          const int o1 = leafi % nl, o2 = (leafi / nl) % nl, o3 = leafi / (nl * nl);
          const int j1 = node % k, j2 = (node / k) % k, j3 = node / (k * k);
          sig[(size_t)g * npb + ((o3 * k + j3) * K + (o2 * k + j2)) * K + (o1 * k + j1)] =
              (R)__ldg(sigma + lv[leafi] * kp + node);
        }
      }
    }
    for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
      const int J = e / n1, m = e - J * n1;
      F1t[(size_t)(g * K + J) * n1 + m] = Ff[((int64_t)(b.mat[0] + J / k) * n1 + m) * k + J % k];
    }
    for (int e = threadIdx.x; e < n1 * K; e += blockDim.x) {
      const int m = e / K, J = e - m * K;
      F2[(size_t)g * n1 * K + e] = Ff[((int64_t)(b.mat[1] + J / k) * n1 + m) * k + J % k];
    }
    for (int e = threadIdx.x; e < kSc * K; e += blockDim.x) {
      const int q = e / K, J = e - q * K;
      Fd[((size_t)g * kSc + q) * K + J] =
          (q < ns) ? Fh[((int64_t)(b.mat[2] + J / k) * nh + s0 + q) * k + J % k] : C{0, 0};
    }
  }
  __syncthreads();
  // stage 1: Z1[q][g][J2][J1] = sum_J3 Fd[g][q][J3] sig[g][J3][J2][J1]
  if (BIG) {
    // one block, sigma from global memory: packed (coalesced along J1), else leaf by leaf
    const int64_t *lv = bleaves + B0.leaf0;
    if (sigp != nullptr) {
      // four columns per thread, two J3 steps per iteration: eight loads in flight
      constexpr int NC = 4;
      const int nth = blockDim.x;
      for (int rem0 = threadIdx.x; rem0 < KK; rem0 += NC * nth) {
        R ar[NC][kSc], ai[NC][kSc];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int q = 0; q < kSc; ++q) ar[c][q] = ai[c][q] = 0;
        const float *sp = sigp + B0.leaf0 * kp + rem0;
        for (int J3 = 0; J3 < K; J3 += 2) {
          R v[2][NC];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < NC; ++c)
              v[h][c] = (J3 + h < K && rem0 + c * nth < KK) ? __ldg(sp + (size_t)(J3 + h) * KK + c * nth) : 0.f;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (J3 + h >= K) break;
#pragma unroll
            for (int q = 0; q < kSc; ++q) {
              const C f = Fd[q * K + J3 + h];
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                ar[c][q] = fmaf(f.x, v[h][c], ar[c][q]);
                ai[c][q] = fmaf(f.y, v[h][c], ai[c][q]);
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (rem0 + c * nth < KK) {
#pragma unroll
            for (int q = 0; q < kSc; ++q) Z1[(size_t)q * KK + rem0 + c * nth] = C{ar[c][q], ai[c][q]};
          }
      }
    }
    for (int rem = threadIdx.x; rem < KK && sigp == nullptr; rem += blockDim.x) {
      R ar[kSc], ai[kSc];
#pragma unroll
      for (int q = 0; q < kSc; ++q) ar[q] = ai[q] = 0;
      {
        const int J2 = rem / K, J1 = rem - J2 * K;
        const int o2 = J2 / k, j2 = J2 - o2 * k, o1 = J1 / k, j1 = J1 - o1 * k;
        for (int o3 = 0; o3 < nl; ++o3) {
          const double *sp = sigma + lv[(o3 * nl + o2) * nl + o1] * kp + j2 * k + j1;
          for (int j3 = 0; j3 < k; ++j3) {
            const R v = (R)__ldg(sp + j3 * k * k);
#pragma unroll
            for (int q = 0; q < kSc; ++q) {
              const C f = Fd[q * K + o3 * k + j3];
              ar[q] = fmaf(f.x, v, ar[q]);
              ai[q] = fmaf(f.y, v, ai[q]);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kSc; ++q) Z1[(size_t)q * KK + rem] = C{ar[q], ai[q]};
    }
  } else {
    for (int e = threadIdx.x; e < G * KK; e += blockDim.x) {
      const int g = e / KK, rem = e - g * KK;
      const R *sp = sig + (size_t)g * npb + rem;
      const C *fp = Fd + (size_t)g * kSc * K;
      R ar[kSc], ai[kSc];
#pragma unroll
      for (int q = 0; q < kSc; ++q) ar[q] = ai[q] = 0;
      for (int J3 = 0; J3 < K; ++J3) {
        const R v = sp[(size_t)J3 * KK];
#pragma unroll
        for (int q = 0; q < kSc; ++q) {
          const C f = fp[q * K + J3];
          ar[q] = fmaf(f.x, v, ar[q]);
          ai[q] = fmaf(f.y, v, ai[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kSc; ++q) Z1[((size_t)q * G + g) * KK + rem] = C{ar[q], ai[q]};
    }
  }
  __syncthreads();
  // stage 2 (CUDA cores, 4 x 4 tiles): Z2[q][m2][g K + J1] = sum_J2 F2[g][m2][J2] Z1[q][g][J2][J1]
  {
    const int tm = (n1 + 3) / 4, tj = (K + 3) / 4, ntile = ns * G * tm * tj;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      int r = t;
      const int bj = r % tj; r /= tj;
      const int bm = r % tm; r /= tm;
      const int g = r % G, q = r / G;
      R ar[4][4], ai[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0;
      const C *fp = F2 + (size_t)g * n1 * K;
      const C *zp = Z1 + ((size_t)q * G + g) * KK;
      for (int J2 = 0; J2 < K; ++J2) {
        C a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = bm * 4 + i;
          a[i] = (m < n1) ? fp[m * K + J2] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int J1 = bj * 4 + j;
          bb[j] = (J1 < K) ? zp[J2 * K + J1] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(ar[i][j], ai[i][j], a[i], bb[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m = bm * 4 + i, J1 = bj * 4 + j;
          if (m < n1 && J1 < K) Z2[((size_t)q * n1 + m) * ldz + g * K + J1] = C{ar[i][j], ai[i][j]};
        }
    }
  }
  __syncthreads();
  // split B operands from F1t: column n < n1p -> real part of output m1 = n, else imaginary part
  for (int e = threadIdx.x; e < NB * 2 * GK; e += blockDim.x) {
    // columns in 16-wide pairs: 8 real-part columns of modes 8 jt .. 8 jt + 7, then their 8
    // imaginary-part columns (so a tile and its partner sit at compile-time indices 2j, 2j+1)
    const int n = e / (2 * GK), kr = e - n * 2 * GK, J = kr >> 1, odd = kr & 1;
    const bool im = ((n >> 3) & 1) != 0;
    const int m1 = (n >> 4) * 8 + (n & 7);
    float v = 0.f;
    if (m1 < n1) {
      const C f = F1t[(size_t)J * n1 + m1];
      v = im ? (odd ? f.x : f.y) : (odd ? -f.y : f.x);
    }
    uint32_t h, l;
    split_tf32(v, h, l);
    Bh[(size_t)n * ldb + kr] = h;
    Bl[(size_t)n * ldb + kr] = l;
  }
  __syncthreads();
  // stage 3 (tensor cores): per plane q and 16-row tile of m2, all 2*n1p output columns
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int mt = (n1 + 15) / 16, nbt = NB / 8, ksteps = (2 * GK) / 8;
  C *out = phi + (int64_t)B0.slot * slot_size;
  for (int job = warp; job < ns * mt; job += blockDim.x >> 5) {
    const int q = job / mt, i0 = (job - q * mt) * 16;
    const float *za = reinterpret_cast<const float *>(Z2 + (size_t)q * n1 * ldz);  // row stride 2 ldz floats
    float acc[NBT][4];
#pragma unroll
    for (int j = 0; j < NBT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int r0 = i0 + gq, r1 = r0 + 8;
    for (int ks = 0; ks < ksteps; ++ks) {
      const int k0 = ks * 8;
      float av[4];
      av[0] = (r0 < n1) ? za[(size_t)r0 * 2 * ldz + k0 + tq] : 0.f;
      av[1] = (r1 < n1) ? za[(size_t)r1 * 2 * ldz + k0 + tq] : 0.f;
      av[2] = (r0 < n1) ? za[(size_t)r0 * 2 * ldz + k0 + tq + 4] : 0.f;
      av[3] = (r1 < n1) ? za[(size_t)r1 * 2 * ldz + k0 + tq + 4] : 0.f;
      uint32_t ah[4], al[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) split_tf32(av[x], ah[x], al[x]);
#pragma unroll
      for (int j = 0; j < NBT; ++j) {
        if (j < nbt) {
          const size_t base = (size_t)(j * 8 + gq) * ldb + k0 + tq;
          mma3(acc[j], ah, al, Bh[base], Bh[base + 4], Bl[base], Bl[base + 4]);
        }
      }
    }
    C *o = out + (int64_t)(s0 + q) * n1 * n1;
#pragma unroll
    for (int j = 0; j < NBT / 2; ++j) {
      if (2 * j < nbt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m2 = h ? r1 : r0;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int m1 = j * 8 + 2 * tq + c;
            if (m2 < n1 && m1 < n1 && FGT_OK_PTR(&o[m2 * n1 + m1])) atomicAdd(&o[m2 * n1 + m1], make_float2(acc[2 * j][2 * h + c], acc[2 * j + 1][2 * h + c]));
          }
        }
      }
    }
  }
}


template <int NBT, bool BIG>  // NBT: n-tiles of 8 output columns held in registers (>= 2 n1p / 8)
__global__ void __launch_bounds__(256, BIG ? 2 : (NBT > 8 ? 2 : 3)) form4_kernel(const Block *__restrict__ blocks, const int32_t *__restrict__ gptr,
                                                    const int64_t *__restrict__ bleaves,
                                                    const double *__restrict__ sigma, const float *__restrict__ sigp,
                                                    const float2 *__restrict__ Ff, const float2 *__restrict__ Fh,
                                                    float2 *__restrict__ phi, int k, int n1, int nh,
                                                    int64_t slot_size) {
  form4_body<NBT, BIG>(blocks, gptr, bleaves, sigma, sigp, Ff, Fh, phi, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- whole-block evaluation

// Stage 2 of the 3D evaluation on the CUDA cores (shared by the whole-block kernels):
// Y2[r][I2][m1] = sum_m2 E2[I2][m2] Y1[r][m2][m1]; 4 x 4 register tiles over (I2, m1) when there
// are enough tiles to occupy the CTA, else one output per thread.
template <typename R>
__device__ __forceinline__ void eval_stage2_3d(const typename C2T<R>::T *__restrict__ Y1,
                                               typename C2T<R>::T *__restrict__ Y2,
                                               const typename C2T<R>::T *__restrict__ E2, int nr, int K, int n1) {
  using C = typename C2T<R>::T;
  const int nn = n1 * n1, tI = (K + 3) / 4, tm = (n1 + 3) / 4;
  if (nr * tI * tm < (int)blockDim.x / 2) {
    for (int e = threadIdx.x; e < nr * K * n1; e += blockDim.x) {
      const int m1 = e % n1, rest = e / n1, I2 = rest % K, r = rest / K;
      const C *ep = E2 + (size_t)I2 * n1;
      const C *yp = Y1 + (size_t)r * nn + m1;
      R ar = 0, ai = 0;
      for (int m2 = 0; m2 < n1; ++m2) cfma(ar, ai, ep[m2], yp[m2 * n1]);
      Y2[e] = C{ar, ai};
    }
  } else {
    const int ntile = nr * tI * tm;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const int bm = t % tm, rest = t / tm, bI = rest % tI, r = rest / tI;
      R ar[4][4], ai[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0;
      const C *yr = Y1 + (size_t)r * nn;
      for (int m2 = 0; m2 < n1; ++m2) {
        C a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int I2 = bI * 4 + i;
          a[i] = (I2 < K) ? E2[(size_t)I2 * n1 + m2] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m1 = bm * 4 + j;
          b[j] = (m1 < n1) ? yr[(size_t)m2 * n1 + m1] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(ar[i][j], ai[i][j], a[i], b[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I2 = bI * 4 + i, m1 = bm * 4 + j;
          if (I2 < K && m1 < n1) Y2[((size_t)r * K + I2) * n1 + m1] = C{ar[i][j], ai[i][j]};
        }
    }
  }
}

// Stage 3 of the 3D evaluation on the CUDA cores: u(r0 + r, I2, I1) = Re sum_m1 E1[I1][m1]
// Y2[r][I2][m1], stored (or added, acc_u) into the block's leaves.
template <typename R>
__device__ __forceinline__ void eval_stage3_3d(const typename C2T<R>::T *__restrict__ Y2,
                                               const typename C2T<R>::T *__restrict__ E1, int nr, int K, int n1,
                                               int r0, int k, int nl, const int64_t *__restrict__ lv,
                                               double *__restrict__ u, bool acc_u) {
  using C = typename C2T<R>::T;
  const int tI = (K + 3) / 4, kp = k * k * k;
  // u(r0 + r, I2, I1) = Re sum_m1 E1[I1][m1] Y2[r][I2][m1]; 4 x 4 register tiles over (I2, I1)
  // when there are enough tiles, else one output per thread
  if (nr * tI * tI < (int)blockDim.x / 2) {
    for (int e = threadIdx.x; e < nr * K * K; e += blockDim.x) {
      const int I1 = e % K, rest = e / K, I2 = rest % K, r = rest / K;
      const C *ep = E1 + (size_t)I1 * n1;
      const C *yp = Y2 + ((size_t)r * K + I2) * n1;
      R acc = 0;
      for (int m1 = 0; m1 < n1; ++m1) {
        const C a = ep[m1], y = yp[m1];
        acc = fma(a.x, y.x, acc);
        acc = fma(-a.y, y.y, acc);
      }
      const int I3 = r0 + r, o1 = I1 / k, o2 = I2 / k, o3 = I3 / k;
      double *up = u + lv[(o3 * nl + o2) * nl + o1] * kp + ((I3 - o3 * k) * k + (I2 - o2 * k)) * k + (I1 - o1 * k);
      if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc); else *up = (double)acc; }
    }
  } else {
    const int ntile = nr * tI * tI;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const int b1 = t % tI, rest = t / tI, b2 = rest % tI, r = rest / tI;
      R acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
      const C *yr = Y2 + (size_t)r * K * n1;
      for (int m1 = 0; m1 < n1; ++m1) {
        C y[4], a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int I2 = b2 * 4 + i;
          y[i] = (I2 < K) ? yr[(size_t)I2 * n1 + m1] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I1 = b1 * 4 + j;
          a[j] = (I1 < K) ? E1[(size_t)I1 * n1 + m1] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] = fma(a[j].x, y[i].x, acc[i][j]);
            acc[i][j] = fma(-a[j].y, y[i].y, acc[i][j]);
          }
      }
      const int I3 = r0 + r, o3 = I3 / k, t3 = I3 - o3 * k;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int I2 = b2 * 4 + i;
        if (I2 >= K) continue;
        const int o2 = I2 / k, t2 = I2 - o2 * k;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I1 = b1 * 4 + j;
          if (I1 >= K) continue;
          const int o1 = I1 / k;
          double *up = u + lv[(o3 * nl + o2) * nl + o1] * kp + (t3 * k + t2) * k + (I1 - o1 * k);
          if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc[i][j]); else *up = (double)acc[i][j]; }
        }
      }
    }
  }
}

// A CTA evaluates KM rows (along the last axis) of one block, all of it when K <= KM: the
// anchor's incoming expansion is read once per CTA (each thread keeps KM accumulators for its
// mode column), then the two remaining contractions run from shared memory.
template <int D, typename R, int KM, bool TC = false>  // TC (FP64, 3D): stages 1-2 on the tensor cores
__device__ __forceinline__ void eval2_body(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const typename C2T<R>::T *__restrict__ Ef,
                                                    const typename C2T<R>::T *__restrict__ Eh,
                                                    const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                    int k, int n1, int nh, int64_t slot_size, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ unsigned char smem_raw[];
  const Block blk = blocks[bx];
  const int K = blk.K, nl = 1 << blk.dl;
  const int r0 = by * KM, nr = min(KM, K - r0);  // rows r0 .. r0 + nr - 1
  if (nr <= 0) return;
  const int RM = min(KM, K);                           // rows the shared arrays are sized for
  const int64_t *lv = bleaves + blk.leaf0;
  const C *ps = psi + (int64_t)blk.slot * slot_size;
  const bool acc_u = (blk.flags & 1) != 0;
  const int nn = (D == 3) ? n1 * n1 : n1;
  C *Y1 = reinterpret_cast<C *>(smem_raw);            // [RM][nn]
  C *Y2 = Y1 + (size_t)RM * nn;                        // [RM][K][n1] (3D)
  C *E1 = Y2 + (D == 3 ? (size_t)RM * K * n1 : 0);     // [K][n1]
  C *E2 = E1 + (size_t)K * n1;                         // [K][n1] (3D)
  C *Ed = E2 + (D == 3 ? (size_t)K * n1 : 0);          // [RM][nh]
  for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
    const int I = e / n1, m = e - I * n1;
    E1[e] = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
    if (D == 3) E2[e] = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
  }
  for (int e = threadIdx.x; e < nr * nh; e += blockDim.x) {
    const int I = r0 + e / nh, m = e % nh;
    Ed[e] = Eh[((int64_t)(blk.mat[D - 1] + I / k) * k + I % k) * nh + m];
  }
  __syncthreads();
  // Y1[r][mode] = sum_{m_d} Ed[r][m_d] psi[m_d][mode]; psi fetched 8 planes at a time so that
  // eight loads are in flight per thread
  if constexpr (TC && sizeof(R) == 8 && D == 3) {
    // one warp per (8 rows, 32 modes): A = Ed, B = psi straight from the slot
    const int mt = (nr + 7) / 8, cb = (nn + 31) / 32;
    for (int job = threadIdx.x >> 5; job < mt * cb; job += blockDim.x >> 5) {
      const int c0 = job % cb, bm = job / cb;
      double acc[8][2];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = 0.0;
      zgemm8_dmma<4>(acc, Ed, nh, nr, bm * 8, ps, nn, nn, c0 * 32, nh);
      const int lane = threadIdx.x & 31, r = bm * 8 + (lane >> 2);
      if (r < nr) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int mode = c0 * 32 + b * 8 + 2 * (lane & 3) + c;
            if (mode < nn) Y1[(size_t)r * nn + mode] = C{acc[2 * b][c], acc[2 * b + 1][c]};
          }
      }
    }
  } else
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    R ar[KM], ai[KM];
#pragma unroll
    for (int r = 0; r < KM; ++r) ar[r] = ai[r] = 0;
    for (int md0 = 0; md0 < nh; md0 += 8) {
      C v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        v[q] = (md0 + q < nh && FGT_OK_PTR(&ps[(int64_t)(md0 + q) * nn + idx])) ? ps[(int64_t)(md0 + q) * nn + idx] : C{0, 0};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (md0 + q < nh) {
#pragma unroll
          for (int r = 0; r < KM; ++r)
            if (r < nr) cfma(ar[r], ai[r], Ed[r * nh + md0 + q], v[q]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < KM; ++r)
      if (r < nr) Y1[(size_t)r * nn + idx] = C{ar[r], ai[r]};
  }
  __syncthreads();
  const int kp = (D == 3) ? k * k * k : k * k;
  if (D == 3) {
    // Y2[r][I2][m1] = sum_m2 E2[I2][m2] Y1[r][m2][m1]
    if constexpr (TC && sizeof(R) == 8) {
      // one warp per (row r, 8 rows of I2, 32 columns of m1): A = E2, B = Y1[r]
      const int mt = (K + 7) / 8, cb = (n1 + 31) / 32;
      for (int job = threadIdx.x >> 5; job < nr * mt * cb; job += blockDim.x >> 5) {
        const int c0 = job % cb, rest = job / cb, bm = rest % mt, r = rest / mt;
        double acc[8][2];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = 0.0;
        zgemm8_dmma<4>(acc, E2, n1, K, bm * 8, Y1 + (size_t)r * nn, n1, n1, c0 * 32, n1);
        const int lane = threadIdx.x & 31, I2 = bm * 8 + (lane >> 2);
        if (I2 < K) {
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const int m1 = c0 * 32 + b * 8 + 2 * (lane & 3) + c;
              if (m1 < n1) Y2[((size_t)r * K + I2) * n1 + m1] = C{acc[2 * b][c], acc[2 * b + 1][c]};
            }
        }
      }
    } else {
      eval_stage2_3d<R>(Y1, Y2, E2, nr, K, n1);
    }
    __syncthreads();
    eval_stage3_3d<R>(Y2, E1, nr, K, n1, r0, k, nl, lv, u, acc_u);
  } else {
    for (int e = threadIdx.x; e < nr * K; e += blockDim.x) {
      const int I1 = e % K, r = e / K;
      const C *ep = E1 + (size_t)I1 * n1;
      const C *yp = Y1 + (size_t)r * nn;
      R acc = 0;
      for (int m1 = 0; m1 < n1; ++m1) {
        const C a = ep[m1], y = yp[m1];
        acc = fma(a.x, y.x, acc);
        acc = fma(-a.y, y.y, acc);
      }
      const int I2 = r0 + r, o1 = I1 / k, o2 = I2 / k;
      double *up = u + lv[o2 * nl + o1] * kp + (I2 - o2 * k) * k + (I1 - o1 * k);
      if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc); else *up = (double)acc; }
    }
  }
}


template <int D, typename R, int KM, bool TC = false>  // TC (FP64, 3D): stages 1-2 on the tensor cores
__global__ void __launch_bounds__(256) eval2_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const typename C2T<R>::T *__restrict__ Ef,
                                                    const typename C2T<R>::T *__restrict__ Eh,
                                                    const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                    int k, int n1, int nh, int64_t slot_size) {
  eval2_body<D, R, KM, TC>(blocks, bleaves, Ef, Eh, psi, u, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- tcgen05 helpers
//
// Fifth-generation tensor cores (sm_100 family): tcgen05.mma reads its operands from shared memory
// through 64-bit matrix descriptors and accumulates in tensor memory (TMEM, 128 lanes x 512
// 32-bit columns per SM), which the CTA allocates, reads back with tcgen05.ld and frees.
// Operand layout used here: K-major without swizzle, 8-row x 16-byte core matrices, the core
// matrices adjacent along K 128 bytes apart (leading byte offset) and the 8-row groups `sbo`
// bytes apart (stride byte offset).

__device__ int g_tc_status;  // set to 1 when a wait on the tensor cores ran out (read by fgt_device_status)


// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, kk) in a K-major operand tile whose 8-row groups are sbo bytes apart.
__device__ __forceinline__ uint32_t umma_off(int row, int kk, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(kk >> 2) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(kk & 3) * 4u;
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}



// Self-test of the time-out path: one thread waits, `clocks` at most, on an mbarrier that nothing
// completes, and sets the status word as the tensor-core kernels do when their waits run out.
__global__ void wait_timeout_selftest_kernel(long long clocks) {
  __shared__ uint64_t bar;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(smem_addr(&bar), 0, clocks)) atomicExch(&g_tc_status, 1);
}



// ----------------------------------------------------------------------------- expansions in tcgen05 operand layout
//
// The incoming expansions, copied once per transform into the A-operand layout of the tcgen05
// evaluation: slot s, tile t (modes q = 128 t .. 128 t + 127, q = m2 n1 + m1), half h (TF32 hi, lo)
// at s * slot_bytes + (2 t + h) * half_bytes, element (row = q - 128 t, kk = 2 m3 + c) at the
// K-major core-matrix offset umma_off(row, kk, 32 kp2); A[q][2 m3] = Re psi[m3][q],
// A[q][2 m3 + 1] = Im psi[m3][q], zero for q >= n1^2 and kk >= 2 nh.  One thread per
// (slot, tile, 4 consecutive kk, row): two complex coefficients, one 16-byte store per half.
__global__ void __launch_bounds__(256) psi_tc_kernel(const float2 *__restrict__ psi, unsigned char *__restrict__ out,
                                                     int n1, int nh, int64_t slot_size, int64_t n_slots) {
  const int nn = n1 * n1, mt = (nn + 127) / 128, kp2 = (2 * nh + 7) / 8 * 8, nq = kp2 / 4;
  const uint32_t sbo = (uint32_t)kp2 * 32, half = 16u * sbo;
  const int64_t per_slot = (int64_t)mt * nq * 128;
  const int64_t total = per_slot * n_slots;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = g / per_slot;
    const int rem = (int)(g - s * per_slot), row = rem & 127, j = (rem >> 7) % nq, t = (rem >> 7) / nq;
    const int q = t * 128 + row;
    const float2 *ps = psi + s * slot_size;
    float2 v0 = make_float2(0.f, 0.f), v1 = v0;
    if (q < nn) {
      if (2 * j < nh) v0 = ps[(int64_t)(2 * j) * nn + q];
      if (2 * j + 1 < nh) v1 = ps[(int64_t)(2 * j + 1) * nn + q];
    }
    uint4 h, l;
    split_tf32(v0.x, h.x, l.x);
    split_tf32(v0.y, h.y, l.y);
    split_tf32(v1.x, h.z, l.z);
    split_tf32(v1.y, h.w, l.w);
    unsigned char *base = out + (size_t)s * ((size_t)mt * 2 * half) + (size_t)(2 * t) * half + umma_off(row, 4 * j, sbo);
    if (FGT_OK_BYTES(base, 16) && FGT_OK_BYTES(base + half, 16)) {
      *reinterpret_cast<uint4 *>(base) = h;
      *reinterpret_cast<uint4 *>(base + half) = l;
    }
  }
}

// ----------------------------------------------------------------------------- evaluation, stage 1 on tcgen05 (3D, FP32)
//
// Whole-block evaluation of KM rows I3 of a block (as eval2_kernel) whose first contraction
//   Y1[r][q] = sum_m3 Ed(I3_r, m3) psi[m3][q],   q = m2 n1 + m1 (nn = n1^2 modes)
// runs on the tensor cores in real form, per tile of 128 modes q:
//   D[q][2r + c] = sum_kk A[q][kk] B[kk][2r + c],   kk = 2 m3 + c'  (c, c' = real, imaginary part),
//   A[q][2 m3] = Re psi, A[q][2 m3 + 1] = Im psi,
//   B[2 m3][2r] = Re Ed, B[2 m3 + 1][2r] = -Im Ed, B[2 m3][2r + 1] = Im Ed, B[2 m3 + 1][2r + 1] = Re Ed,
// each operand split into TF32 hi and lo halves and the product taken as lo*hi + hi*lo + hi*hi
// (3xTF32, FP32-accurate), accumulated in FP32 in TMEM (one 128 x N accumulator per tile,
// N = max(16, 2 KM)).  A comes from the operand copy of the expansion (psi_tc_kernel): thread 0
// streams its half-tiles through a ring of kEval6Ring shared buffers with bulk asynchronous copies
// (a full and an empty mbarrier per buffer), issues the MMAs of each half as it lands and commits
// them to the buffer's empty barrier, keeping two copies in flight ahead of the tensor cores.
// The other threads build B and the E1 / E2 matrices meanwhile, then everyone reads the
// accumulators back and stages 2-3 run from shared memory on the CUDA cores (eval_stage2_3d /
// eval_stage3_3d).  A wait that runs out sets g_tc_status, skips the rest of the block and frees
// the tensor memory.
template <int KM>
__global__ void __launch_bounds__(256) eval6_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const float2 *__restrict__ Ef, const float2 *__restrict__ Eh,
                                                    const unsigned char *__restrict__ psi_tc, double *__restrict__ u,
                                                    int k, int n1, int nh, int tmem_cols) {
  constexpr int N = KM <= 8 ? 16 : 2 * KM, S = kEval6Ring;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Block blk = blocks[blockIdx.x];
  const int K = blk.K, nl = 1 << blk.dl;
  const int r0 = blockIdx.y * KM, nr = min(KM, K - r0);
  if (nr <= 0) return;
  const int RM = min(KM, K);
  const int64_t *lv = bleaves + blk.leaf0;
  const bool acc_u = (blk.flags & 1) != 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nn = n1 * n1, mt = (nn + 127) / 128, nst = 2 * mt;  // stages: (tile, half)
  const int kp2 = (2 * nh + 7) / 8 * 8, ksteps = kp2 / 8;
  const uint32_t sbo = (uint32_t)kp2 * 32, half_b = 16u * sbo;
  const unsigned char *src = psi_tc + (size_t)blk.slot * ((size_t)nst * half_b);
  // shared memory: ring [S] half-tiles, B hi, B lo | overlaid by Y1 after stage 1; Y2, E1, E2, words
  unsigned char *ring = smem_raw;
  unsigned char *bh = ring + (size_t)S * half_b, *bl = bh + (size_t)N * kp2 * 4;
  const size_t stage_b = (size_t)S * half_b + 2 * (size_t)N * kp2 * 4, y1_b = 8 * (size_t)RM * nn;
  const size_t r1 = ((stage_b > y1_b ? stage_b : y1_b) + 127) & ~(size_t)127;
  float2 *Y1 = reinterpret_cast<float2 *>(smem_raw);
  float2 *Y2 = reinterpret_cast<float2 *>(smem_raw + r1);
  float2 *E1 = Y2 + (size_t)RM * K * n1;
  float2 *E2 = E1 + (size_t)K * n1;
  uint64_t *full = reinterpret_cast<uint64_t *>(E2 + (size_t)K * n1);  // [S]
  uint64_t *empty = full + S;                                          // [S]
  uint32_t *tslot = reinterpret_cast<uint32_t *>(empty + S);
  if (tid == 0) {
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(empty + b)), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the first S - 1 copies start before anything else
  if (tid == 0)
    for (int i = 0; i < S - 1 && i < nst; ++i)
      bulk_copy_g2s(smem_addr(ring + (size_t)i * half_b), src + (size_t)i * half_b, half_b, smem_addr(full + i));
  for (int e = tid; e < K * n1; e += blockDim.x) {
    const int I = e / n1, m = e - I * n1;
    E1[e] = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
    E2[e] = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
  }
  // B operand: rows n = 2r + c (N of them, rows of absent output rows zero), K-major over kk
  for (int e = tid; e < N * kp2; e += blockDim.x) {
    const int n = e / kp2, kk = e - n * kp2, r = n >> 1, m3 = kk >> 1;
    float v = 0.f;
    if (r < nr && m3 < nh) {
      const int I = r0 + r;
      const float2 ed = Eh[((int64_t)(blk.mat[2] + I / k) * k + I % k) * nh + m3];
      v = (n & 1) ? ((kk & 1) ? ed.x : ed.y) : ((kk & 1) ? -ed.y : ed.x);
    }
    uint32_t hi, lo;
    split_tf32(v, hi, lo);
    const uint32_t o = umma_off(n, kk, sbo);
    *reinterpret_cast<uint32_t *>(bh + o) = hi;
    *reinterpret_cast<uint32_t *>(bl + o) = lo;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B, written by these threads, read by the MMAs
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool fail = false, drained = true;
  if (tid == 0) {
    // producer of the copies and issuer of the MMAs: stage i = (tile i / 2, half i % 2) in buffer i % S
    const uint32_t idesc = umma_idesc_tf32(128, N), sbh = smem_addr(bh), sbl = smem_addr(bl);
    int issued = min(S - 1, nst), committed = -1;
    for (int i = 0; i < nst; ++i) {
      const int b = i % S;
      if (!mbar_wait(smem_addr(full + b), (uint32_t)((i / S) & 1))) { fail = true; break; }
      tc_fence_after();
      const int t = i >> 1;
      const uint32_t d = tmem + (uint32_t)(t * N), sa = smem_addr(ring + (size_t)b * half_b);
      for (int s = 0; s < ksteps; ++s) {
        const uint32_t ko = (uint32_t)s * 256u;  // two core matrices along K per MMA (K = 8)
        if ((i & 1) == 0) {                      // hi half of A: hi * lo, hi * hi
          umma_tf32(d, umma_desc(sa + ko, sbo), umma_desc(sbl + ko, sbo), idesc, s > 0);
          umma_tf32(d, umma_desc(sa + ko, sbo), umma_desc(sbh + ko, sbo), idesc, 1);
        } else {                                 // lo half of A: lo * hi
          umma_tf32(d, umma_desc(sa + ko, sbo), umma_desc(sbh + ko, sbo), idesc, 1);
        }
      }
      umma_commit(smem_addr(empty + b));
      committed = i;
      const int j = i + S - 1;  // next copy, into the buffer stage i - 1 read (its MMAs run behind these)
      if (j < nst) {
        const int bj = j % S;
        if (j >= S && !mbar_wait(smem_addr(empty + bj), (uint32_t)((j / S - 1) & 1))) { fail = true; break; }
        bulk_copy_g2s(smem_addr(ring + (size_t)bj * half_b), src + (size_t)j * half_b, half_b, smem_addr(full + bj));
        issued = j + 1;
      }
    }
    if (!fail) {
      if (!mbar_wait(smem_addr(empty + (nst - 1) % S), (uint32_t)(((nst - 1) / S) & 1))) fail = true;
    } else {
      // give the copies and MMAs still in flight a bounded chance to land before the exit; if one
      // of these waits runs out as well, an asynchronous copy or MMA may still land after this CTA
      // has freed its shared and tensor memory, which status 2 reports
      for (int i = max(committed + 1, issued - S); i < issued; ++i)
        if (i >= 0 && !mbar_wait(smem_addr(full + i % S), (uint32_t)((i / S) & 1))) drained = false;
      if (committed >= 0 && !mbar_wait(smem_addr(empty + committed % S), (uint32_t)((committed / S) & 1)))
        drained = false;
    }
  }
  if (__syncthreads_or(fail)) {
    if (tid == 0) atomicMax(&g_tc_status, drained ? 1 : 2);
    fail = true;
  }
  tc_fence_after();
  if (!fail) {
    // read the accumulators back: warp w holds TMEM lanes 32 (w % 4) .. + 31, columns
    // (w / 4) N/2 .. + N/2 - 1, i.e. rows r = (w / 4) N/4 .. + N/4 - 1 of its modes
    constexpr int HC = N / 2;
    const int c0 = (warp >> 2) * HC;
    for (int t = 0; t < mt; ++t) {
      uint32_t v[HC];
      const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(t * N + c0);
      if constexpr (HC == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(addr));
      } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(addr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int q = t * 128 + 32 * (warp & 3) + lane;
      if (q < nn) {
#pragma unroll
        for (int j = 0; j < HC / 2; ++j) {
          const int r = c0 / 2 + j;
          if (r < nr) Y1[(size_t)r * nn + q] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  if (fail) return;
  eval_stage2_3d<float>(Y1, Y2, E2, nr, K, n1);
  __syncthreads();
  eval_stage3_3d<float>(Y2, E1, nr, K, n1, r0, k, nl, lv, u, acc_u);
}

// ----------------------------------------------------------------------------- evaluation, all contractions on tcgen05 (3D, FP32)
//
// u(I3, I2, I1) = Re sum_{m3 >= 0} Eh(I3, m3) sum_m2 E2(I2, m2) sum_m1 E1(I1, m1) psi[m3][m2][m1]
// (Lemma thm:pweval) as three chained real GEMMs on the fifth-generation tensor cores, one CTA per
// block of K = 8, 16 or 32 nodes per axis, every product in 3xTF32 (lo*hi + hi*lo + hi*hi of
// TF32 halves, FP32 accumulators in tensor memory).  The expansion is stored padded for this
// kernel ("eval7 layout", written by the gather): slot s holds [m3][m2 < 32][m1 < 32] complex
// values, zero beyond n1, so that one tile of 128 rows (m3, m2) x 64 floats (m1, re/im) is a
// tensor-map box.  Per chunk of 128/K planes m3:
//   stage 1  D1[(m3, m2)][(I1, c)]   = sum_{(m1, c')} psi[(m3, m2)][(m1, c')] B1[(I1, c)][(m1, c')]
//            A from the tensor map (cp.async.bulk.tensor, 128-byte swizzle, two 32-float slabs per
//            tile through a double buffer), split into TF32 halves in place;
//   stage 2  D2[(m3, I1)][(I2, c)]   = sum_{(m2, c')} A2[(m3, I1)][(m2, c')] B2[(I2, c)][(m2, c')]
//            A2 written from D1 by the CUDA cores (tcgen05.ld, split, swizzled stores);
//   stage 3  D3[(I2, I1)][I3]       += sum_{(m3, c')} A3[(I2, I1)][(m3, c')] B3[I3][(m3, c')]
//            A3 written from D2, B3 = (Re Eh, -Im Eh): the real part only, accumulated over chunks.
// B1 / B2 are the real forms of E1 / E2 (rows (I, c) = Re / Im of the product, columns (m, c')),
// built once per CTA from the FP32 matrices.  Thread 0 issues the tensor-map copies and the MMAs;
// every wait is bounded and, when one runs out, the CTA drains what it has in flight (bounded),
// sets the status word (1, or 2 when the drain ran out too), frees its tensor memory and returns.
namespace e7 {
constexpr int kP = 32;    // padded modes per full-range axis (n1 <= 32)
__host__ __device__ constexpr int cm3(int K) { return 128 / K; }          // planes m3 per chunk
__host__ __device__ constexpr int n12(int K) { return 2 * K; }            // N of stages 1 and 2
__host__ __device__ constexpr int n3(int K) { return K < 16 ? 16 : K; }   // N of stage 3
__host__ __device__ constexpr int kd3(int K) { return 256 / K; }          // stage-3 K per chunk (floats)
__host__ __device__ constexpr int t3(int K) { return K * K > 128 ? K * K / 128 : 1; }  // stage-3 M tiles
constexpr int kKB3 = 32;  // stage-3 contraction over all chunks (2 nh <= 32 floats)
__host__ __device__ constexpr size_t off_a23() { return 65536; }
__host__ __device__ constexpr size_t off_b1() { return 131072; }
__host__ __device__ constexpr size_t b12_bytes(int K) { return 512u * (size_t)n12(K); }  // 2 slabs, hi + lo
__host__ __device__ constexpr size_t off_b2(int K) { return off_b1() + b12_bytes(K); }
__host__ __device__ constexpr size_t off_b3(int K) { return off_b2(K) + b12_bytes(K); }
__host__ __device__ constexpr size_t off_bar(int K) { return off_b3(K) + 256u * (size_t)n3(K); }
__host__ __device__ constexpr size_t smem_bytes(int K) { return off_bar(K) + 64 + 1024; }  // 7 barriers, the
                                                                                           // TMEM slot, alignment
__host__ __device__ constexpr int tmem_cols(int K) {
  return (2 * kP + n12(K) + t3(K) * n3(K)) <= 128 ? 128 : (2 * kP + n12(K) + t3(K) * n3(K)) <= 256 ? 256 : 512;
}
}  // namespace e7

__device__ int g_tc7_status;  // status word of eval7_kernel (same meaning as g_tc_status)

// K-major operand with 128-byte swizzle (the layout of a tensor-map box of 32 floats x rows with
// CU_TENSOR_MAP_SWIZZLE_128B): slabs of 32 floats along K, each rows x 128 bytes; in an 8-row atom
// of 1024 bytes the 16-byte chunk j of row r sits at chunk j ^ (r mod 8).
__device__ __forceinline__ uint32_t sw128_off(int row, int kk, int rows) {
  const int slab = kk >> 5, f = kk & 31;
  return (uint32_t)slab * (uint32_t)rows * 128u + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
         ((uint32_t)((f >> 2) ^ (row & 7)) << 4) + (uint32_t)(f & 3) * 4u;
}

__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset: unused with the 128-byte swizzle along K
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                 // descriptor version of the sm_100 family
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar,
                                            uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}


// hi / lo TF32 halves of a pair, stored at byte offset o of the hi and lo operand copies
__device__ __forceinline__ void put_split2(unsigned char *hi, unsigned char *lo, uint32_t o, float a, float b) {
  uint32_t h0, l0, h1, l1;
  split_tf32(a, h0, l0);
  split_tf32(b, h1, l1);
  *reinterpret_cast<uint2 *>(hi + o) = make_uint2(h0, h1);
  *reinterpret_cast<uint2 *>(lo + o) = make_uint2(l0, l1);
}

template <int K, int NW>  // NW warps: 4 per TMEM lane quarter x NW / 4 column shares
__global__ void __launch_bounds__(NW * 32, 1) eval7_kernel(const __grid_constant__ CUtensorMap psi_map,
                                                       const Block *__restrict__ blocks,
                                                       const int64_t *__restrict__ bleaves,
                                                       const float2 *__restrict__ Ef, const float2 *__restrict__ Eh,
                                                       double *__restrict__ u, int k, int n1, int nh) {
  using namespace e7;
  constexpr int N12 = n12(K), N3 = n3(K), CM3 = cm3(K), KD3 = kd3(K), T3 = t3(K), R3 = 128 * T3;
  constexpr int TPC = CM3 / (128 / kP);  // stage-1 tiles (128 / kP planes each) per chunk
  // accumulator columns a warp reads back: NW / 4 warps share each TMEM lane quarter
  constexpr int CQ = NW / 4, C1 = 2 * kP / CQ, C2 = N12 / CQ, C3 = N3 / CQ;
  constexpr int TC = tmem_cols(K);
  constexpr uint32_t SLAB = 16384;       // one 128-row x 128-byte slab
  constexpr uint32_t SBO3 = (uint32_t)(KD3 / 4) * 128u, SBO3B = (uint32_t)(kKB3 / 4) * 128u;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t sb = smem_addr(sm);
  const Block blk = blocks[blockIdx.x];
  const int nl = 1 << blk.dl;
  const int64_t *lv = bleaves + blk.leaf0;
  const bool acc_u = (blk.flags & 1) != 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3, hh = warp >> 2;  // hh: column quarter
  const int nch = (nh + CM3 - 1) / CM3, nloads = nch * TPC * 2;
  // mbarriers: full[2] (copies landed), empty[2] (stage-1 MMAs of a buffer done), mma2, mma3 (one
  // commit per chunk each), drain (used once, after a time-out)
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + off_bar(K));
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 7);
  const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + 2), mma2 = smem_addr(bars + 4),
                 mma3 = smem_addr(bars + 5), drainb = smem_addr(bars + 6);
  unsigned char *a23h = sm + off_a23(), *a2l = a23h + 2 * SLAB, *a3l = a23h + (size_t)R3 * KD3 * 4;
  unsigned char *b1h = sm + off_b1(), *b1l = b1h + 256 * N12;
  unsigned char *b2h = sm + off_b2(K), *b2l = b2h + 256 * N12;
  unsigned char *b3h = sm + off_b3(K), *b3l = b3h + 128 * N3;
  if (tid == 0) {
    for (int b = 0; b < 7; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&psi_map)) : "memory");
  }
  __syncthreads();
  // load i: chunk i / (2 TPC), tile (i / 2) % TPC of the chunk, slab i % 2, into buffer i % 2
  auto issue = [&](int i) {
    const int j = i / (2 * TPC), tl = (i >> 1) % TPC, s = i & 1;
    const int t = j * TPC + tl;
    tma_load_3d(sb + (uint32_t)(i & 1) * 2 * SLAB, &psi_map, 32 * s, 128 * t, blk.slot, full0 + 8 * (i & 1), SLAB);
  };
  if (tid == 0) {
    issue(0);
    if (nloads > 1) issue(1);
  }
  // B operands from the block's 1D matrices (real forms, TF32 halves)
  for (int e = tid; e < K * kP; e += blockDim.x) {  // (I, m): both c rows, both c' columns
    const int I = e / kP, m = e - I * kP;
    float2 e1 = make_float2(0.f, 0.f), e2 = e1;
    if (m < n1) {
      e1 = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
      e2 = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
    }
    if (I < K) {
      put_split2(b1h, b1l, sw128_off(2 * I, 2 * m, N12), e1.x, -e1.y);
      put_split2(b1h, b1l, sw128_off(2 * I + 1, 2 * m, N12), e1.y, e1.x);
      put_split2(b2h, b2l, sw128_off(2 * I, 2 * m, N12), e2.x, -e2.y);
      put_split2(b2h, b2l, sw128_off(2 * I + 1, 2 * m, N12), e2.y, e2.x);
    }
  }
  for (int e = tid; e < N3 * (kKB3 / 2); e += blockDim.x) {  // (I3, m3)
    const int I = e / (kKB3 / 2), m = e - I * (kKB3 / 2);
    float2 eh = make_float2(0.f, 0.f);
    if (I < K && m < nh) eh = Eh[((int64_t)(blk.mat[2] + I / k) * k + I % k) * nh + m];
    put_split2(b3h, b3l, umma_off(I, 2 * m, SBO3B), eh.x, -eh.y);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)), "r"(TC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot, tD1 = tmem, tD2 = tmem + 2 * kP, tD3 = tmem + 2 * kP + N12;
  const uint32_t id12 = umma_idesc_tf32(128, N12), id3 = umma_idesc_tf32(128, N3);
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  int issued = nloads < 2 ? nloads : 2;  // loads issued so far (thread 0)
  int n3c = 0;                           // stage-3 commits issued (thread 0)
  bool fail = false;
  // thread 0: issue load x into buffer x % 2 once the MMAs of load x - 2 (the buffer's previous
  // contents) are done; loads are issued in order, each once
  auto refill = [&](int x) -> bool {
    if (x >= nloads || x != issued) return true;
    if (x >= 2 && !mbar_wait(empty0 + 8 * (x & 1), (uint32_t)(((x - 2) >> 1) & 1))) return false;
    issue(x);
    issued = x + 1;
    return true;
  };
  int i = 0;
  for (int j = 0; j < nch && !fail; ++j) {
    // ---- stage 1: the chunk's tiles, two slabs each
    for (int tl = 0; tl < TPC && !fail; ++tl) {
      for (int s = 0; s < 2; ++s, ++i) {
        const int b = i & 1;
        // the other buffer's next load, while this one is split (its MMAs, of load i - 1, run meanwhile)
        bool ok = tid != 0 || refill(i + 1);
        ok = ok && mbar_wait(full0 + 8 * b, (uint32_t)((i >> 1) & 1));
        if (__syncthreads_or(!ok)) { fail = true; break; }
        uint4 *hp = reinterpret_cast<uint4 *>(sm + (size_t)b * 2 * SLAB), *lp = hp + SLAB / 16;
        for (int e = tid; e < (int)(SLAB / 16); e += blockDim.x) {
          const uint4 v = hp[e];
          uint4 hv, lw;
          split_tf32(__uint_as_float(v.x), hv.x, lw.x);
          split_tf32(__uint_as_float(v.y), hv.y, lw.y);
          split_tf32(__uint_as_float(v.z), hv.z, lw.z);
          split_tf32(__uint_as_float(v.w), hv.w, lw.w);
          hp[e] = hv;
          lp[e] = lw;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
          const uint32_t ah = sb + (uint32_t)b * 2 * SLAB, al = ah + SLAB;
          const uint32_t bh = smem_addr(b1h) + (uint32_t)s * N12 * 128u, bl = smem_addr(b1l) + (uint32_t)s * N12 * 128u;
          const uint32_t d = tD1 + (uint32_t)(tl * N12);
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = (uint32_t)ks * 32u;
            umma_tf32(d, umma_desc_sw128(ah + o), umma_desc_sw128(bl + o), id12, (s > 0 || ks > 0) ? 1u : 0u);
            umma_tf32(d, umma_desc_sw128(ah + o), umma_desc_sw128(bh + o), id12, 1u);
            umma_tf32(d, umma_desc_sw128(al + o), umma_desc_sw128(bh + o), id12, 1u);
          }
          umma_commit(empty0 + 8 * b);
        }
      }
    }
    if (fail) break;
    // ---- stage 1 done (the commit of the chunk's last load covers all earlier MMAs)
    {
      const int il = i - 1;
      bool ok = mbar_wait(empty0 + 8 * (il & 1), (uint32_t)((il >> 1) & 1));
      if (tid == 0 && ok) ok = refill(il + 2);  // the next chunk's first copy runs during stages 2-3
      if (__syncthreads_or(!ok)) { fail = true; break; }
    }
    tc_fence_after();
    {  // D1 -> A2: warp (q, hh) reads lanes 32q.. (rows (m3, m2)), its share of the 64 columns
      uint32_t v[C1];
      tmem_ld<C1>(tD1 + lane_base + (uint32_t)(C1 * hh), v);
      const int l = 32 * q + lane, m2 = l & (kP - 1), mrow = l / kP;
#pragma unroll
      for (int p = 0; p < C1 / 2; ++p) {
        const int col = C1 * hh + 2 * p, tl = col / N12, I1 = (col - tl * N12) >> 1;
        const int m3l = tl * (128 / kP) + mrow;
        put_split2(a23h, a2l, sw128_off(m3l * K + I1, 2 * m2, 128), __uint_as_float(v[2 * p]),
                   __uint_as_float(v[2 * p + 1]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {  // ---- stage 2
      const uint32_t ah = smem_addr(a23h), al = smem_addr(a2l), bh = smem_addr(b2h), bl = smem_addr(b2l);
      for (int ks = 0; ks < 8; ++ks) {
        const uint32_t oa = (uint32_t)(ks >> 2) * SLAB + (uint32_t)(ks & 3) * 32u;
        const uint32_t ob = (uint32_t)(ks >> 2) * N12 * 128u + (uint32_t)(ks & 3) * 32u;
        umma_tf32(tD2, umma_desc_sw128(ah + oa), umma_desc_sw128(bl + ob), id12, ks > 0 ? 1u : 0u);
        umma_tf32(tD2, umma_desc_sw128(ah + oa), umma_desc_sw128(bh + ob), id12, 1u);
        umma_tf32(tD2, umma_desc_sw128(al + oa), umma_desc_sw128(bh + ob), id12, 1u);
      }
      umma_commit(mma2);
    }
    {
      const bool ok = mbar_wait(mma2, (uint32_t)(j & 1));
      if (__syncthreads_or(!ok)) { fail = true; break; }
    }
    tc_fence_after();
    {  // D2 -> A3 (over A2, whose MMAs are done): lanes = rows (m3, I1), columns (I2, c) of share hh
      uint32_t v[C2];
      tmem_ld<C2>(tD2 + lane_base + (uint32_t)(C2 * hh), v);
      const int l = 32 * q + lane, m3l = l / K, I1 = l - m3l * K;
#pragma unroll
      for (int p = 0; p < C2 / 2; ++p) {
        const int I2 = hh * (C2 / 2) + p;
        put_split2(a23h, a3l, umma_off(I2 * K + I1, 2 * m3l, SBO3), __uint_as_float(v[2 * p]),
                   __uint_as_float(v[2 * p + 1]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {  // ---- stage 3, accumulated over the chunks
      const uint32_t ah = smem_addr(a23h), al = smem_addr(a3l), bh = smem_addr(b3h), bl = smem_addr(b3l);
      for (int t = 0; t < T3; ++t)
        for (int ks = 0; ks < KD3 / 8; ++ks) {
          const uint32_t oa = (uint32_t)t * 16u * SBO3 + (uint32_t)ks * 256u;
          const uint32_t ob = (uint32_t)(j * (KD3 / 4) + 2 * ks) * 128u;
          const uint32_t d = tD3 + (uint32_t)(t * N3), acc = (j > 0 || ks > 0) ? 1u : 0u;
          umma_tf32(d, umma_desc(ah + oa, SBO3), umma_desc(bl + ob, SBO3B), id3, acc);
          umma_tf32(d, umma_desc(ah + oa, SBO3), umma_desc(bh + ob, SBO3B), id3, 1u);
          umma_tf32(d, umma_desc(al + oa, SBO3), umma_desc(bh + ob, SBO3B), id3, 1u);
        }
      umma_commit(mma3);
      ++n3c;
    }
  }
  if (!fail) {
    const bool ok = mbar_wait(mma3, (uint32_t)((nch - 1) & 1));
    if (__syncthreads_or(!ok)) fail = true;
  }
  if (fail) {
    // drain (bounded) what may still be in flight: copies not yet waited for, the last MMAs
    bool drained = true;
    if (tid == 0) {
      for (int x = i; x < issued; ++x)
        if (!mbar_wait(full0 + 8 * (x & 1), (uint32_t)((x >> 1) & 1), 1LL << 28)) drained = false;
      // one commit on a barrier of its own after everything issued: its completion covers every
      // earlier MMA of this thread
      umma_commit(drainb);
      if (!mbar_wait(drainb, 0u, 1LL << 28)) drained = false;
      atomicMax(&g_tc7_status, drained ? 1 : 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC));
    return;
  }
  tc_fence_after();
  // ---- D3 -> u, tile by tile (128 rows (I2, I1) = RI2 values of I2 x all I1): the accumulators are
  // widened to FP64 on the integer pipes and staged in shared memory (the free copy ring) as
  // [I3][I2 of the tile][I1], then written in runs of RI2 k consecutive values of u (one leaf row
  // block per (o1, I3)) with 16-byte stores.  The block's leaves' offsets into u sit in shared memory.
  constexpr int RI2 = 128 / K < K ? 128 / K : K;  // I2 values per tile
  double *stage = reinterpret_cast<double *>(sm);   // K * RI2 * K values: at most 32 KB
  int64_t *lofs = reinterpret_cast<int64_t *>(sm + 32768);
  const int kp3 = k * k * k;
  for (int e = tid; e < nl * nl * nl; e += blockDim.x) lofs[e] = lv[e] * kp3;
  __syncthreads();
#pragma unroll 1
  for (int t = 0; t < T3; ++t) {
    {
      uint32_t v[C3];
      tmem_ld<C3>(tD3 + lane_base + (uint32_t)(t * N3 + hh * C3), v);
      const int rl = 32 * q + lane;  // row within the tile: I2l = rl / K, I1 = rl % K
      if (rl < RI2 * K) {
#pragma unroll
        for (int x = 0; x < C3; ++x) {
          const int I3 = hh * C3 + x;
          if (I3 < K) stage[I3 * (RI2 * K) + rl] = f32_to_f64_int(v[x]);
        }
      }
    }
    __syncthreads();
    // runs: (I3, o1) -> RI2 rows of k values (I2l, i1), contiguous in u within a leaf; pairs of
    // values per thread.  k and nl are powers of two here (K = nl k = 8, 16, 32, k even): shifts.
    const int I2base = t * RI2, lk = __ffs(k) - 1, lnl = blk.dl, lr = __ffs(RI2) - 1 + lk;
    const int npairs = (K * nl * RI2 * k) >> 1;
    for (int e = tid; e < npairs; e += blockDim.x) {
      const int pe = 2 * e, run = pe >> lr, w = pe & ((1 << lr) - 1);
      const int I3 = run >> lnl, o1 = run & (nl - 1), I2l = w >> lk, i1 = w & (k - 1);
      const int o3 = I3 >> lk, I2 = I2base + I2l, o2 = I2 >> lk;
      const double2 vv = *reinterpret_cast<const double2 *>(stage + I3 * (RI2 * K) + I2l * K + (o1 << lk) + i1);
      const double v0 = vv.x, v1 = vv.y;
      double *up = u + lofs[(((o3 << lnl) + o2) << lnl) + o1] + ((((I3 & (k - 1)) << lk) + (I2 & (k - 1))) << lk) + i1;
      if (acc_u) {
        if (FGT_OK_PTR(up)) atomicAdd(up, v0);
        if (FGT_OK_PTR(up + 1)) atomicAdd(up + 1, v1);
      } else if (FGT_OK_BYTES(up, 16)) {
        *reinterpret_cast<double2 *>(up) = make_double2(v0, v1);
      }
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC));
}

// ----------------------------------------------------------------------------- form, all contractions on tcgen05 (3D, FP32)
//
// phi[m3][m2][m1] (+)= sum_{J3, J2, J1} Fh(m3, J3) F2(m2, J2) F1(m1, J1) sigma(J3, J2, J1)  (Lemma pwbox),
// one CTA per block of K = 8, 16 or 32 nodes per axis, every product in 3xTF32 with FP32
// accumulators in tensor memory, contracted x3 first (into the half-range axis), then x2, then x1:
//   stage 1  D1[(J1, J2)][(m3, c)]  = sum_J3 sigma[(J1, J2)][J3] B1[(m3, c)][J3]        (B1 = Re / Im Fh)
//            A from the packed FP32 density (rows (J1, J2) of K values, J3 fastest) through a tensor
//            map with the swizzle of a K-float row (32, 64 or 128 bytes), split into TF32 halves in place;
//   stage 2  D2[(J1, m3)][(m2, c)]  = sum_{(J2, c')} A2[(J1, m3)][(J2, c')] B2[(m2, c)][(J2, c')]
//   stage 3  D3[(m2, m3)][(m1, c)] += sum_{(J1, c')} A3[(m2, m3)][(J1, c')] B3[(m1, c)][(J1, c')]
// in chunks of 8 planes J1 (A2, A3 written from D1, D2 by the CUDA cores), D3 accumulated over the
// chunks and written to the anchor's slot: stored when the block is its anchor's only one (flags
// bit 1), added atomically otherwise.  Waits, time-outs and the status word as in eval7_kernel.
namespace f7 {
constexpr int kP = 32;    // padded modes per full-range axis (n1 <= 32); m3 < 16
__host__ __device__ constexpr uint32_t a1_bytes(int K) { return 128u * (uint32_t)K * 4u; }  // one stage-1 tile
__host__ __device__ constexpr int tpc(int K) { return K >= 16 ? K / 16 : 1; }               // tiles per chunk
__host__ __device__ constexpr int nchunk(int K) { return K / 8; }                             // chunks of 8 J1
__host__ __device__ constexpr int kd2(int K) { return 2 * K < 32 ? 32 : 2 * K; }            // stage-2 K, padded
__host__ __device__ constexpr size_t off_a23(int K) { return 4 * (size_t)a1_bytes(K); }     // ring: 2 x (hi, lo)
__host__ __device__ constexpr size_t off_b1(int K) { return off_a23(K) + 65536; }
__host__ __device__ constexpr size_t off_b2(int K) { return off_b1(K) + 256u * (size_t)K; }
__host__ __device__ constexpr size_t off_b3(int K) { return off_b2(K) + 512u * (size_t)kd2(K); }
__host__ __device__ constexpr size_t off_bar(int K) { return off_b3(K) + 1024u * (size_t)K; }
__host__ __device__ constexpr size_t smem_bytes(int K) { return off_bar(K) + 64 + 1024; }
constexpr int kTmemCols = 512;  // D1 (64), D2 (64), D3 (4 tiles x 64)
}  // namespace f7

// Descriptor of a K-major operand with a 32-, 64- or 128-byte swizzle (rows of 8, 16 or 32 floats,
// 8-row atoms), as a tensor map with the matching swizzle leaves it.
__device__ __forceinline__ uint64_t umma_desc_swz(uint32_t saddr, int row_floats) {
  const uint32_t rb = (uint32_t)row_floats * 4u;
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(((8u * rb) >> 4) & 0x3FFF) << 32;  // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(row_floats == 8 ? 6 : row_floats == 16 ? 4 : 2) << 61;  // 32-, 64-, 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar,
                                            uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ int g_tcf_status;  // status word of form7_kernel (same meaning as g_tc_status)

template <int K, int NW>  // NW warps: 4 per TMEM lane quarter x NW / 4 column shares
__global__ void __launch_bounds__(NW * 32, 1) form7_kernel(const __grid_constant__ CUtensorMap sig_map,
                                                       const Block *__restrict__ blocks,
                                                       const float2 *__restrict__ Ff, const float2 *__restrict__ Fh,
                                                       float2 *__restrict__ phi, int k, int n1, int nh,
                                                       int64_t slot_size) {
  using namespace f7;
  constexpr int TPC = tpc(K), NCH = nchunk(K), KD2 = kd2(K), NL = NCH * TPC;
  // accumulator columns a warp reads back: NW / 4 warps share each TMEM lane quarter
  constexpr int CQ = NW / 4, C1 = 32 / CQ, C2 = 64 / CQ;
  constexpr uint32_t A1 = a1_bytes(K);
  constexpr uint32_t SBOB1 = (uint32_t)(K / 4) * 128u, SBO3 = 4u * 128u, SBOB3 = (uint32_t)(2 * K / 4) * 128u;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const uint32_t sb = smem_addr(sm);
  const Block blk = blocks[blockIdx.x];
  const bool sole = (blk.flags & 2) != 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3, hh = warp >> 2;
  const int row0 = (int)(blk.leaf0 * (int64_t)(k * k * k) / K);  // the block's first K-float row
  // mbarriers: full[2], empty[2], mma2, mma3, drain
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + off_bar(K));
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 7);
  const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + 2), mma2 = smem_addr(bars + 4),
                 mma3 = smem_addr(bars + 5), drainb = smem_addr(bars + 6);
  unsigned char *a23h = sm + off_a23(K), *a2l = a23h + (size_t)128 * KD2 * 4, *a3l = a23h + 512u * 16u * 4u;
  unsigned char *b1h = sm + off_b1(K), *b1l = b1h + 128u * K;
  unsigned char *b2h = sm + off_b2(K), *b2l = b2h + 256u * KD2;
  unsigned char *b3h = sm + off_b3(K), *b3l = b3h + 512u * K;
  if (tid == 0) {
    for (int b = 0; b < 7; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&sig_map)) : "memory");
  }
  __syncthreads();
  auto issue = [&](int i) {  // stage-1 tile i (rows row0 + 128 i) into buffer i % 2
    tma_load_2d(sb + (uint32_t)(i & 1) * 2u * A1, &sig_map, 0, row0 + 128 * i, full0 + 8 * (i & 1), A1);
  };
  if (tid == 0) {
    issue(0);
    if (NL > 1) issue(1);
  }
  // A2 / A3 region zeroed once (the padding columns of A2 for K = 8 are never written)
  for (int e = tid; e < 65536 / 16; e += blockDim.x) reinterpret_cast<uint4 *>(a23h)[e] = make_uint4(0, 0, 0, 0);
  // B operands (real forms of the block's 1D form matrices, TF32 halves)
  for (int e = tid; e < 16 * K; e += blockDim.x) {  // B1[(m3, c)][J3]
    const int m = e / K, J = e - m * K;
    float2 f = make_float2(0.f, 0.f);
    if (m < nh) f = Fh[((int64_t)(blk.mat[2] + J / k) * nh + m) * k + J % k];
    uint32_t h0, l0, h1, l1;
    split_tf32(f.x, h0, l0);
    split_tf32(f.y, h1, l1);
    *reinterpret_cast<uint32_t *>(b1h + umma_off(2 * m, J, SBOB1)) = h0;
    *reinterpret_cast<uint32_t *>(b1l + umma_off(2 * m, J, SBOB1)) = l0;
    *reinterpret_cast<uint32_t *>(b1h + umma_off(2 * m + 1, J, SBOB1)) = h1;
    *reinterpret_cast<uint32_t *>(b1l + umma_off(2 * m + 1, J, SBOB1)) = l1;
  }
  for (int e = tid; e < kP * (KD2 / 2); e += blockDim.x) {  // B2[(m2, c)][(J2, c')], B3[(m1, c)][(J1, c')]
    const int m = e / (KD2 / 2), J = e - m * (KD2 / 2);
    float2 f2 = make_float2(0.f, 0.f), f1 = f2;
    if (m < n1 && J < K) {
      f2 = Ff[((int64_t)(blk.mat[1] + J / k) * n1 + m) * k + J % k];
      f1 = Ff[((int64_t)(blk.mat[0] + J / k) * n1 + m) * k + J % k];
    }
    put_split2(b2h, b2l, sw128_off(2 * m, 2 * J, 2 * kP), f2.x, -f2.y);
    put_split2(b2h, b2l, sw128_off(2 * m + 1, 2 * J, 2 * kP), f2.y, f2.x);
    if (J < K) {
      put_split2(b3h, b3l, umma_off(2 * m, 2 * J, SBOB3), f1.x, -f1.y);
      put_split2(b3h, b3l, umma_off(2 * m + 1, 2 * J, SBOB3), f1.y, f1.x);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot, tD1 = tmem, tD2 = tmem + 64, tD3 = tmem + 128;
  const uint32_t id1 = umma_idesc_tf32(128, 32), id2 = umma_idesc_tf32(128, 64);
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  int issued = NL < 2 ? NL : 2;
  bool fail = false;
  auto refill = [&](int x) -> bool {
    if (x >= NL || x != issued) return true;
    if (x >= 2 && !mbar_wait(empty0 + 8 * (x & 1), (uint32_t)(((x - 2) >> 1) & 1))) return false;
    issue(x);
    issued = x + 1;
    return true;
  };
  int i = 0;
  for (int c = 0; c < NCH && !fail; ++c) {
    // ---- stage 1: the chunk's tiles
    for (int tl = 0; tl < TPC; ++tl, ++i) {
      const int b = i & 1;
      bool ok = tid != 0 || refill(i + 1);
      ok = ok && mbar_wait(full0 + 8 * b, (uint32_t)((i >> 1) & 1));
      if (__syncthreads_or(!ok)) { fail = true; break; }
      uint4 *hp = reinterpret_cast<uint4 *>(sm + (size_t)b * 2 * A1), *lp = hp + A1 / 16;
      for (int e = tid; e < (int)(A1 / 16); e += blockDim.x) {
        const uint4 v = hp[e];
        uint4 hv, lw;
        split_tf32(__uint_as_float(v.x), hv.x, lw.x);
        split_tf32(__uint_as_float(v.y), hv.y, lw.y);
        split_tf32(__uint_as_float(v.z), hv.z, lw.z);
        split_tf32(__uint_as_float(v.w), hv.w, lw.w);
        hp[e] = hv;
        lp[e] = lw;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint32_t ah = sb + (uint32_t)b * 2u * A1, al = ah + A1, bh = smem_addr(b1h), bl = smem_addr(b1l);
        const uint32_t d = tD1 + (uint32_t)(tl * 32);
        for (int ks = 0; ks < K / 8; ++ks) {
          const uint32_t oa = (uint32_t)ks * 32u, ob = (uint32_t)ks * 256u;
          umma_tf32(d, umma_desc_swz(ah + oa, K), umma_desc(bl + ob, SBOB1), id1, ks > 0 ? 1u : 0u);
          umma_tf32(d, umma_desc_swz(ah + oa, K), umma_desc(bh + ob, SBOB1), id1, 1u);
          umma_tf32(d, umma_desc_swz(al + oa, K), umma_desc(bh + ob, SBOB1), id1, 1u);
        }
        umma_commit(empty0 + 8 * b);
      }
    }
    if (fail) break;
    {  // stage 1 of the chunk done; the next chunk's first copy starts
      const int il = i - 1;
      bool ok = mbar_wait(empty0 + 8 * (il & 1), (uint32_t)((il >> 1) & 1));
      if (tid == 0 && ok) ok = refill(il + 2);
      if (__syncthreads_or(!ok)) { fail = true; break; }
    }
    tc_fence_after();
    // ---- D1 -> A2: lanes = rows (J1, J2) of the chunk's tiles, columns (m3, c) of half hh
#pragma unroll 1
    for (int tl = 0; tl < TPC; ++tl) {
      const int rc = tl * 128 + 32 * q;  // first row of this warp's lanes within the chunk
      if (rc >= 8 * K) continue;         // K = 8: the tile's second half holds no rows of the block
      uint32_t v[C1];
      tmem_ld<C1>(tD1 + lane_base + (uint32_t)(tl * 32 + C1 * hh), v);
      const int r = rc + lane, J1l = r / K, J2 = r - J1l * K;
#pragma unroll
      for (int p = 0; p < C1 / 2; ++p) {
        const int m3 = (C1 / 2) * hh + p;
        put_split2(a23h, a2l, sw128_off(J1l * 16 + m3, 2 * J2, 128), __uint_as_float(v[2 * p]),
                   __uint_as_float(v[2 * p + 1]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {  // ---- stage 2
      const uint32_t ah = smem_addr(a23h), al = smem_addr(a2l), bh = smem_addr(b2h), bl = smem_addr(b2l);
      for (int ks = 0; ks < KD2 / 8; ++ks) {
        const uint32_t oa = (uint32_t)(ks >> 2) * 16384u + (uint32_t)(ks & 3) * 32u;
        const uint32_t ob = (uint32_t)(ks >> 2) * 8192u + (uint32_t)(ks & 3) * 32u;
        umma_tf32(tD2, umma_desc_sw128(ah + oa), umma_desc_sw128(bl + ob), id2, ks > 0 ? 1u : 0u);
        umma_tf32(tD2, umma_desc_sw128(ah + oa), umma_desc_sw128(bh + ob), id2, 1u);
        umma_tf32(tD2, umma_desc_sw128(al + oa), umma_desc_sw128(bh + ob), id2, 1u);
      }
      umma_commit(mma2);
    }
    {
      const bool ok = mbar_wait(mma2, (uint32_t)(c & 1));
      if (__syncthreads_or(!ok)) { fail = true; break; }
    }
    tc_fence_after();
    {  // ---- D2 -> A3: lanes = rows (J1, m3), columns (m2, c) of quarter hh
      uint32_t v[C2];
      tmem_ld<C2>(tD2 + lane_base + (uint32_t)(C2 * hh), v);
      const int l = 32 * q + lane, J1l = l >> 4, m3 = l & 15;
#pragma unroll
      for (int p = 0; p < C2 / 2; ++p) {
        const int m2 = (C2 / 2) * hh + p;
        put_split2(a23h, a3l, umma_off(m2 * 16 + m3, 2 * J1l, SBO3), __uint_as_float(v[2 * p]),
                   __uint_as_float(v[2 * p + 1]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {  // ---- stage 3, accumulated over the chunks
      const uint32_t ah = smem_addr(a23h), al = smem_addr(a3l), bh = smem_addr(b3h), bl = smem_addr(b3l);
      for (int t = 0; t < 4; ++t)
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t oa = (uint32_t)t * 16u * SBO3 + (uint32_t)ks * 256u;
          const uint32_t ob = (uint32_t)(4 * c + 2 * ks) * 128u;
          const uint32_t d = tD3 + (uint32_t)(t * 64), acc = (c > 0 || ks > 0) ? 1u : 0u;
          umma_tf32(d, umma_desc(ah + oa, SBO3), umma_desc(bl + ob, SBOB3), id2, acc);
          umma_tf32(d, umma_desc(ah + oa, SBO3), umma_desc(bh + ob, SBOB3), id2, 1u);
          umma_tf32(d, umma_desc(al + oa, SBO3), umma_desc(bh + ob, SBOB3), id2, 1u);
        }
      umma_commit(mma3);
    }
    {  // A3 is overwritten by the next chunk's A2
      const bool ok = mbar_wait(mma3, (uint32_t)(c & 1));
      if (__syncthreads_or(!ok)) { fail = true; break; }
    }
  }
  if (fail) {
    bool drained = true;
    if (tid == 0) {
      for (int x = i; x < issued; ++x)
        if (!mbar_wait(full0 + 8 * (x & 1), (uint32_t)((x >> 1) & 1), 1LL << 28)) drained = false;
      umma_commit(drainb);
      if (!mbar_wait(drainb, 0u, 1LL << 28)) drained = false;
      atomicMax(&g_tcf_status, drained ? 1 : 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    return;
  }
  tc_fence_after();
  // ---- D3 -> phi: lanes = rows (m2, m3), columns (m1, c) of half hh
  float2 *out = phi + (int64_t)blk.slot * slot_size;
#pragma unroll 1
  for (int t = 0; t < 4; ++t) {
    uint32_t v[C2];
    tmem_ld<C2>(tD3 + lane_base + (uint32_t)(t * 64 + C2 * hh), v);
    const int row = t * 128 + 32 * q + lane, m2 = row >> 4, m3 = row & 15;
    if (m2 < n1 && m3 < nh) {
      float2 *o = out + ((int64_t)m3 * n1 + m2) * n1;
#pragma unroll
      for (int p = 0; p < C2 / 2; ++p) {
        const int m1 = (C2 / 2) * hh + p;
        if (m1 < n1 && FGT_OK_PTR(o + m1)) {
          const float2 val = make_float2(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
          if (sole) o[m1] = val;
          else atomicAdd(o + m1, val);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ----------------------------------------------------------------------------- evaluation, half-range axis last (3D)
//
// u(I3, I2, I1) = Re sum_{m3 >= 0} Eh(I3, m3) sum_m2 E2(I2, m2) sum_m1 E1(I1, m1) psi[m3][m2][m1]
// contracted m1 first and the half-range axis m3 last: K nh n1^2 + K^2 nh n1 + K^3 nh complex
// products (the last one real-valued) instead of K nh n1^2 + K^2 n1^2 + K^3 n1 with m3 first --
// 18 % (K = 8) to 39 % (K = 32) fewer at n1 = 2 nh - 1.  A CTA takes RC rows I1 of a block:
//   stage 1: T1[r][m3][m2] = sum_m1 E1(I1_r, m1) psi[m3][m2][m1]   (one thread per (m3, m2) row)
//   stage 2: T2[r][I2][m3] = sum_m2 E2(I2, m2) T1[r][m3][m2]       (4 x 4 register tiles)
//   stage 3: u = Re sum_m3 Eh(I3, m3) T2[r][I2][m3]                (4 x 4 register tiles)
template <typename R, int RC>
__device__ __forceinline__ void eval5_body(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const typename C2T<R>::T *__restrict__ Ef,
                                                    const typename C2T<R>::T *__restrict__ Eh,
                                                    const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                    int k, int n1, int nh, int64_t slot_size, int bx, int by) {
  using C = typename C2T<R>::T;
  extern __shared__ __align__(16) unsigned char smem_e5[];
  const Block blk = blocks[bx];
  const int K = blk.K, nl = 1 << blk.dl;
  const int i0 = by * RC, nr = min(RC, K - i0);  // rows I1 = i0 .. i0 + nr - 1
  if (nr <= 0) return;
  const int64_t *lv = bleaves + blk.leaf0;
  const C *ps = psi + (int64_t)blk.slot * slot_size;
  const bool acc_u = (blk.flags & 1) != 0;
  const int nrow = nh * n1;                             // (m3, m2) rows of the slot
  C *T1 = reinterpret_cast<C *>(smem_e5);               // [RC][nh][n1]
  C *T2 = T1 + (size_t)RC * nrow;                       // [RC][K][nh]
  C *E1 = T2 + (size_t)RC * K * nh;                     // [RC][n1]  (rows I1 of the chunk)
  C *E2 = E1 + (size_t)RC * n1;                         // [K][n1]
  C *Ez = E2 + (size_t)K * n1;                          // [K][nh]   (last axis, m3 >= 0)
  for (int e = threadIdx.x; e < nr * n1; e += blockDim.x) {
    const int I = i0 + e / n1, m = e % n1;
    E1[e] = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
  }
  for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
    const int I = e / n1, m = e - I * n1;
    E2[e] = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
  }
  for (int e = threadIdx.x; e < K * nh; e += blockDim.x) {
    const int I = e / nh, m = e - I * nh;
    Ez[e] = Eh[((int64_t)(blk.mat[2] + I / k) * k + I % k) * nh + m];
  }
  __syncthreads();
  // stage 1: each thread one (m3, m2) row of the slot, RC accumulators
  for (int row = threadIdx.x; row < nrow; row += blockDim.x) {
    const C *pr = ps + (int64_t)row * n1;
    R ar[RC], ai[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) ar[r] = ai[r] = 0;
    for (int m0 = 0; m0 < n1; m0 += 4) {
      C v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = (m0 + q < n1) ? pr[m0 + q] : C{0, 0};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (m0 + q >= n1) break;
#pragma unroll
        for (int r = 0; r < RC; ++r)
          if (r < nr) cfma(ar[r], ai[r], E1[r * n1 + m0 + q], v[q]);
      }
    }
#pragma unroll
    for (int r = 0; r < RC; ++r)
      if (r < nr) T1[(size_t)r * nrow + row] = C{ar[r], ai[r]};
  }
  __syncthreads();
  // stage 2: T2[r][I2][m3] = sum_m2 E2[I2][m2] T1[r][m3][m2]; 4 x 4 tiles over (I2, m3)
  {
    const int tI = (K + 3) / 4, tm = (nh + 3) / 4, ntile = nr * tI * tm;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const int bm = t % tm, rest = t / tm, bI = rest % tI, r = rest / tI;
      R ar[4][4], ai[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0;
      const C *t1 = T1 + (size_t)r * nrow;
      for (int m2 = 0; m2 < n1; ++m2) {
        C a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int I2 = bI * 4 + i;
          a[i] = (I2 < K) ? E2[(size_t)I2 * n1 + m2] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m3 = bm * 4 + j;
          b[j] = (m3 < nh) ? t1[(size_t)m3 * n1 + m2] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(ar[i][j], ai[i][j], a[i], b[j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I2 = bI * 4 + i, m3 = bm * 4 + j;
          if (I2 < K && m3 < nh) T2[((size_t)r * K + I2) * nh + m3] = C{ar[i][j], ai[i][j]};
        }
    }
  }
  __syncthreads();
  // stage 3: u(I3, I2, I1) = Re sum_m3 Ez[I3][m3] T2[r][I2][m3]; 4 x 4 tiles over (I3, I2)
  {
    const int kp = k * k * k, tI = (K + 3) / 4, ntile = nr * tI * tI;
    for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
      const int b2 = t % tI, rest = t / tI, b3 = rest % tI, r = rest / tI;
      R acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
      const C *t2 = T2 + (size_t)r * K * nh;
      for (int m3 = 0; m3 < nh; ++m3) {
        C a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int I3 = b3 * 4 + i;
          a[i] = (I3 < K) ? Ez[(size_t)I3 * nh + m3] : C{0, 0};
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I2 = b2 * 4 + j;
          b[j] = (I2 < K) ? t2[(size_t)I2 * nh + m3] : C{0, 0};
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] = fma(a[i].x, b[j].x, acc[i][j]);
            acc[i][j] = fma(-a[i].y, b[j].y, acc[i][j]);
          }
      }
      const int I1 = i0 + r, o1 = I1 / k, t1 = I1 - o1 * k;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int I3 = b3 * 4 + i;
        if (I3 >= K) continue;
        const int o3 = I3 / k, t3 = I3 - o3 * k;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int I2 = b2 * 4 + j;
          if (I2 >= K) continue;
          const int o2 = I2 / k, t2i = I2 - o2 * k;
          double *up = u + lv[(o3 * nl + o2) * nl + o1] * kp + (t3 * k + t2i) * k + t1;
          if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc[i][j]); else *up = (double)acc[i][j]; }
        }
      }
    }
  }
}


template <typename R, int RC>
__global__ void __launch_bounds__(256) eval5_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const typename C2T<R>::T *__restrict__ Ef,
                                                    const typename C2T<R>::T *__restrict__ Eh,
                                                    const typename C2T<R>::T *__restrict__ psi, double *__restrict__ u,
                                                    int k, int n1, int nh, int64_t slot_size) {
  eval5_body<R, RC>(blocks, bleaves, Ef, Eh, psi, u, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- tensor-core evaluation, stages 2-3 (3D, FP32)
//
// eval2_kernel's work split (KM rows of a block per CTA, psi read once in stage 1 on the CUDA
// cores), with the two contractions that follow on the tensor cores in 3xTF32:
//   stage 2, per row r: Y2[r] (K x n1) = E2 (K x n1) Y1[r] (n1 x n1), complex, embedded as a real
//     product over the interleaved (re, im) index of m2 (A = E2, B = Y1[r]);
//   stage 3, per row r: u[r] (K x K) = Re Y2[r] (K x n1) E1^T (n1 x K): only the real part, so B
//     carries (Re E1, -Im E1) on the interleaved index of m1.
// One warp per (row, 16-row tile); operands are split into TF32 hi / lo as they are loaded.
template <int NBT, int KM>  // NBT: n-tiles of 8 stage-2 columns in registers (>= 2 ceil(n1/8)); KM rows per CTA
__device__ __forceinline__ void eval4_body(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const float2 *__restrict__ Ef, const float2 *__restrict__ Eh,
                                                    const float2 *__restrict__ psi, double *__restrict__ u, int k,
                                                    int n1, int nh, int64_t slot_size, int bx, int by) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_e4[];
  const Block blk = blocks[bx];
  const int K = blk.K, nl = 1 << blk.dl;
  const int r0 = by * KM, nr = min(KM, K - r0);
  if (nr <= 0) return;
  const int RM = min(KM, K);
  const int64_t *lv = bleaves + blk.leaf0;
  const C *ps = psi + (int64_t)blk.slot * slot_size;
  const bool acc_u = (blk.flags & 1) != 0;
  const int nn = n1 * n1;
  C *Y1 = reinterpret_cast<C *>(smem_e4);              // [RM][nn]
  C *Y2 = Y1 + (size_t)RM * nn;                         // [RM][K][n1]
  C *E1 = Y2 + (size_t)RM * K * n1;                     // [K][n1]
  C *E2 = E1 + (size_t)K * n1;                          // [K][n1]
  C *Ed = E2 + (size_t)K * n1;                          // [RM][nh]
  for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
    const int I = e / n1, m = e - I * n1;
    E1[e] = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
    E2[e] = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
  }
  for (int e = threadIdx.x; e < nr * nh; e += blockDim.x) {
    const int I = r0 + e / nh, m = e % nh;
    Ed[e] = Eh[((int64_t)(blk.mat[2] + I / k) * k + I % k) * nh + m];
  }
  __syncthreads();
  // stage 1 (CUDA cores): Y1[r][mode] = sum_m3 Ed[r][m3] psi[m3][mode], 8 planes in flight
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    float ar[KM], ai[KM];
#pragma unroll
    for (int r = 0; r < KM; ++r) ar[r] = ai[r] = 0.f;
    for (int md0 = 0; md0 < nh; md0 += 8) {
      C v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (md0 + q < nh) ? ps[(int64_t)(md0 + q) * nn + idx] : C{0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (md0 + q < nh) {
#pragma unroll
          for (int r = 0; r < KM; ++r)
            if (r < nr) cfma(ar[r], ai[r], Ed[r * nh + md0 + q], v[q]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < KM; ++r)
      if (r < nr) Y1[(size_t)r * nn + idx] = C{ar[r], ai[r]};
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt = (K + 15) / 16, kst = (2 * n1 + 7) / 8, nbt = 2 * ((n1 + 7) / 8);
  // stage 2: per (r, 16-row tile of I2), all 2 * ceil(n1/8) column tiles (re / im pairs)
  for (int job = warp; job < nr * mt; job += nwarp) {
    const int r = job / mt, i0 = (job - r * mt) * 16;
    const C *y1 = Y1 + (size_t)r * nn;
    float acc[NBT][4];
#pragma unroll
    for (int j = 0; j < NBT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int ra = i0 + g, rb = ra + 8;
    for (int ks = 0; ks < kst; ++ks) {
      // real index k0 + t and k0 + t + 4 -> complex m2 = k0/2 + (t>>1) (+2), part t & 1
      const int mA = ks * 4 + (t >> 1), mB = mA + 2, part = t & 1;
      float av[4];
      {
        const C e0 = (ra < K && mA < n1) ? E2[(size_t)ra * n1 + mA] : C{0.f, 0.f};
        const C e1 = (rb < K && mA < n1) ? E2[(size_t)rb * n1 + mA] : C{0.f, 0.f};
        const C e2 = (ra < K && mB < n1) ? E2[(size_t)ra * n1 + mB] : C{0.f, 0.f};
        const C e3 = (rb < K && mB < n1) ? E2[(size_t)rb * n1 + mB] : C{0.f, 0.f};
        av[0] = part ? e0.y : e0.x;
        av[1] = part ? e1.y : e1.x;
        av[2] = part ? e2.y : e2.x;
        av[3] = part ? e3.y : e3.x;
      }
      uint32_t ah[4], al[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) split_tf32(av[x], ah[x], al[x]);
#pragma unroll
      for (int jj = 0; jj < NBT / 2; ++jj) {
        if (2 * jj >= nbt) break;
        const int m1 = jj * 8 + g;
        const C y0 = (mA < n1 && m1 < n1) ? y1[(size_t)mA * n1 + m1] : C{0.f, 0.f};
        const C y4 = (mB < n1 && m1 < n1) ? y1[(size_t)mB * n1 + m1] : C{0.f, 0.f};
        uint32_t bh0, bl0, bh1, bl1;
        // real-part tile: (Re, -Im) on the interleaved index
        split_tf32(part ? -y0.y : y0.x, bh0, bl0);
        split_tf32(part ? -y4.y : y4.x, bh1, bl1);
        mma3(acc[2 * jj], ah, al, bh0, bh1, bl0, bl1);
        // imaginary-part tile: (Im, Re)
        split_tf32(part ? y0.x : y0.y, bh0, bl0);
        split_tf32(part ? y4.x : y4.y, bh1, bl1);
        mma3(acc[2 * jj + 1], ah, al, bh0, bh1, bl0, bl1);
      }
    }
    C *y2 = Y2 + (size_t)r * K * n1;
#pragma unroll
    for (int jj = 0; jj < NBT / 2; ++jj) {
      if (2 * jj >= nbt) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = h ? rb : ra;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int m1 = jj * 8 + 2 * t + c;
          if (row < K && m1 < n1) y2[(size_t)row * n1 + m1] = C{acc[2 * jj][2 * h + c], acc[2 * jj + 1][2 * h + c]};
        }
      }
    }
  }
  __syncthreads();
  // stage 3: u(r0 + r, I2, I1) = Re sum_m1 Y2[r][I2][m1] E1[I1][m1]; per (r, 16-row tile of I2)
  const int kp = k * k * k, ntk = (K + 7) / 8;
  for (int job = warp; job < nr * mt; job += nwarp) {
    const int r = job / mt, i0 = (job - r * mt) * 16;
    const C *y2 = Y2 + (size_t)r * K * n1;
    float acc[4][4];  // K <= 32: at most 4 column tiles
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int ra = i0 + g, rb = ra + 8;
    for (int ks = 0; ks < kst; ++ks) {
      const int mA = ks * 4 + (t >> 1), mB = mA + 2, part = t & 1;
      float av[4];
      {
        const C e0 = (ra < K && mA < n1) ? y2[(size_t)ra * n1 + mA] : C{0.f, 0.f};
        const C e1 = (rb < K && mA < n1) ? y2[(size_t)rb * n1 + mA] : C{0.f, 0.f};
        const C e2 = (ra < K && mB < n1) ? y2[(size_t)ra * n1 + mB] : C{0.f, 0.f};
        const C e3 = (rb < K && mB < n1) ? y2[(size_t)rb * n1 + mB] : C{0.f, 0.f};
        av[0] = part ? e0.y : e0.x;
        av[1] = part ? e1.y : e1.x;
        av[2] = part ? e2.y : e2.x;
        av[3] = part ? e3.y : e3.x;
      }
      uint32_t ah[4], al[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) split_tf32(av[x], ah[x], al[x]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= ntk) break;
        const int I1 = j * 8 + g;
        const C f0 = (mA < n1 && I1 < K) ? E1[(size_t)I1 * n1 + mA] : C{0.f, 0.f};
        const C f4 = (mB < n1 && I1 < K) ? E1[(size_t)I1 * n1 + mB] : C{0.f, 0.f};
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(part ? -f0.y : f0.x, bh0, bl0);
        split_tf32(part ? -f4.y : f4.x, bh1, bl1);
        mma3(acc[j], ah, al, bh0, bh1, bl0, bl1);
      }
    }
    const int I3 = r0 + r, o3 = I3 / k, t3 = I3 - o3 * k;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= ntk) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int I2 = h ? rb : ra;
        if (I2 >= K) continue;
        const int o2 = I2 / k, t2 = I2 - o2 * k;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int I1 = j * 8 + 2 * t + c;
          if (I1 >= K) continue;
          const int o1 = I1 / k;
          double *up = u + lv[(o3 * nl + o2) * nl + o1] * kp + (t3 * k + t2) * k + (I1 - o1 * k);
          const double v = (double)acc[j][2 * h + c];
          if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, v); else *up = v; }
        }
      }
    }
  }
}


template <int NBT, int KM>  // NBT: n-tiles of 8 stage-2 columns in registers (>= 2 ceil(n1/8)); KM rows per CTA
__global__ void __launch_bounds__(256) eval4_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const float2 *__restrict__ Ef, const float2 *__restrict__ Eh,
                                                    const float2 *__restrict__ psi, double *__restrict__ u, int k,
                                                    int n1, int nh, int64_t slot_size) {
  eval4_body<NBT, KM>(blocks, bleaves, Ef, Eh, psi, u, k, n1, nh, slot_size, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------------------- tensor-core evaluation (3D, FP32)
//
// eval2_kernel with its first contraction, Y1 (K x n1^2) = Ed (K x nh) psi (nh x n1^2), on the
// tensor cores in 3xTF32: Ed is the A operand (16 rows, kept in registers for the whole CTA),
// psi streams in as B fragments straight from the slot, 8 mode columns per tile.
// A CTA evaluates rows [8 y, 8 y + 8) of one block (K <= 16), so that its shared memory
// (Y1 for 8 rows) leaves room for two or more CTAs per SM.
constexpr int kEvalRows = 8;

template <int KST>  // k-steps of 8 over the interleaved 2 nh contraction: 2 nh <= 8 KST
__global__ void __launch_bounds__(256) eval3_kernel(const Block *__restrict__ blocks, const int64_t *__restrict__ bleaves,
                                                    const float2 *__restrict__ Ef, const float2 *__restrict__ Eh,
                                                    const float2 *__restrict__ psi, double *__restrict__ u, int k,
                                                    int n1, int nh, int64_t slot_size) {
  using R = float;
  using C = float2;
  extern __shared__ unsigned char smem_raw[];
  const Block blk = blocks[blockIdx.x];
  const int K = blk.K, nl = 1 << blk.dl;
  const int rbase = blockIdx.y * kEvalRows;
  if (rbase >= K) return;
  const int RB = min(kEvalRows, K - rbase);
  const int64_t *lv = bleaves + blk.leaf0;
  const C *ps = psi + (int64_t)blk.slot * slot_size;
  const bool acc_u = (blk.flags & 1) != 0;
  const int nn = n1 * n1;
  C *Y1 = reinterpret_cast<C *>(smem_raw);            // [RB][nn]
  C *Y2 = Y1 + (size_t)kEvalRows * nn;                 // [RB][K][n1]
  C *E1 = Y2 + (size_t)kEvalRows * K * n1;             // [K][n1]
  C *E2 = E1 + (size_t)K * n1;                         // [K][n1]
  C *Ed = E2 + (size_t)K * n1;                         // [RB][nh]
  for (int e = threadIdx.x; e < K * n1; e += blockDim.x) {
    const int I = e / n1, m = e - I * n1;
    E1[e] = Ef[((int64_t)(blk.mat[0] + I / k) * k + I % k) * n1 + m];
    E2[e] = Ef[((int64_t)(blk.mat[1] + I / k) * k + I % k) * n1 + m];
  }
  for (int e = threadIdx.x; e < RB * nh; e += blockDim.x) {
    const int I = rbase + e / nh, m = e % nh;
    Ed[e] = Eh[((int64_t)(blk.mat[2] + I / k) * k + I % k) * nh + m];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gq = lane >> 2, tq = lane & 3;
  const int ksteps = (2 * nh + 7) / 8;
  // A operand: row gq of this CTA's Ed rows (rows 8..15 of the tile are zero), interleaved
  // (re, im) contraction index; kept in registers for the whole CTA
  uint32_t ah[KST][4], al[KST][4];
#pragma unroll
  for (int ks = 0; ks < KST; ++ks) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int kr = ks * 8 + tq + ((x & 2) ? 4 : 0), md = kr >> 1;
      float v = 0.f;
      if (!(x & 1) && ks < ksteps && gq < RB && md < nh) {
        const C e = Ed[gq * nh + md];
        v = (kr & 1) ? e.y : e.x;
      }
      split_tf32(v, ah[ks][x], al[ks][x]);
    }
  }
  const int ntiles = (nn + 7) / 8;
  for (int tile = warp; tile < ntiles; tile += blockDim.x >> 5) {
    const int p = tile * 8 + gq;  // this lane's B column (mode index)
    float cre[4] = {0.f, 0.f, 0.f, 0.f}, cim[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < KST; ++ks) {
      if (ks < ksteps) {
        const int md0 = (ks * 8 + tq) >> 1, md1 = md0 + 2, odd = tq & 1;
        const C v0 = (p < nn && md0 < nh) ? ps[(int64_t)md0 * nn + p] : C{0.f, 0.f};
        const C v1 = (p < nn && md1 < nh) ? ps[(int64_t)md1 * nn + p] : C{0.f, 0.f};
        uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
        split_tf32(odd ? -v0.y : v0.x, rh0, rl0);
        split_tf32(odd ? -v1.y : v1.x, rh1, rl1);
        split_tf32(odd ? v0.x : v0.y, ih0, il0);
        split_tf32(odd ? v1.x : v1.y, ih1, il1);
        mma3(cre, ah[ks], al[ks], rh0, rh1, rl0, rl1);
        mma3(cim, ah[ks], al[ks], ih0, ih1, il0, il1);
      }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {  // rows gq (c0, c1); rows gq + 8 are padding
      const int col = tile * 8 + 2 * tq + x;
      if (gq < RB && col < nn) Y1[(size_t)gq * nn + col] = C{cre[x], cim[x]};
    }
  }
  __syncthreads();
  const int kp = k * k * k;
  // Y2[r][I2][m1] = sum_m2 E2[I2][m2] Y1[r][m2][m1]
  for (int e = threadIdx.x; e < RB * K * n1; e += blockDim.x) {
    const int m1 = e % n1, rest = e / n1, I2 = rest % K, r = rest / K;
    const C *ep = E2 + (size_t)I2 * n1;
    const C *yp = Y1 + (size_t)r * nn + m1;
    R ar = 0, ai = 0;
    for (int m2 = 0; m2 < n1; ++m2) cfma(ar, ai, ep[m2], yp[m2 * n1]);
    Y2[e] = C{ar, ai};
  }
  __syncthreads();
  // u(rbase + r, I2, I1) = Re sum_m1 E1[I1][m1] Y2[r][I2][m1]
  for (int e = threadIdx.x; e < RB * K * K; e += blockDim.x) {
    const int I1 = e % K, rest = e / K, I2 = rest % K, r = rest / K, rg = rbase + r;
    const C *ep = E1 + (size_t)I1 * n1;
    const C *yp = Y2 + ((size_t)r * K + I2) * n1;
    R acc = 0;
    for (int m1 = 0; m1 < n1; ++m1) {
      const C a = ep[m1], y = yp[m1];
      acc = fmaf(a.x, y.x, acc);
      acc = fmaf(-a.y, y.y, acc);
    }
    const int o1 = I1 / k, o2 = I2 / k, o3 = rg / k;
    double *up = u + lv[(o3 * nl + o2) * nl + o1] * kp + ((rg - o3 * k) * k + (I2 - o2 * k)) * k + (I1 - o1 * k);
    if (FGT_OK_PTR(up)) { if (acc_u) atomicAdd(up, (double)acc); else *up = (double)acc; }
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
// Each thread handles kGatherMpt modes, blockDim apart (coalesced), sharing the per-source
// bookkeeping; a CTA covers kGatherMpt * blockDim consecutive modes of one anchor.
constexpr int kGatherMpt = 4;

template <int D, typename R>
__device__ __forceinline__ void gather_body(const int32_t *__restrict__ dst, const int64_t *__restrict__ ptr,
                              const GatherSrc *__restrict__ src, const typename C2T<R>::T *__restrict__ Pf,
                              const typename C2T<R>::T *__restrict__ Ph, const typename C2T<R>::T *__restrict__ phi,
                              typename C2T<R>::T *__restrict__ psi, int n1, int nh, int64_t slot_size,
                              int psi_pitch, int bx, int by) {
  using C = typename C2T<R>::T;
  constexpr int MPT = kGatherMpt;
  const int i = bx;
  const int64_t base = (int64_t)by * blockDim.x * MPT + threadIdx.x;
  int m1[MPT], m2[MPT], m3[MPT];
  bool ok[MPT];
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    const int64_t idx = base + (int64_t)j * blockDim.x;
    ok[j] = idx < slot_size;
    mode_index<D>(ok[j] ? idx : 0, n1, m1[j], m2[j], m3[j]);
  }
  // factors of the second and last axes (the last axis stores m >= 0 only)
  const C *P2 = (D == 3) ? Pf : Ph;
  const int s2 = (D == 3) ? n1 : nh;
  R a1r[MPT], a1i[MPT], a2r[MPT], a2i[MPT], a3r[MPT], a3i[MPT];
#pragma unroll
  for (int j = 0; j < MPT; ++j) a1r[j] = a1i[j] = a2r[j] = a2i[j] = a3r[j] = a3i[j] = 0;
  int g1 = -1, g2 = -1;  // current (o_2, o_3) run and o_3 run
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const GatherSrc g = src[q];
    const int run1 = g.code / 3, run2 = g.code / 9;
    if (run1 != g1) {
      if (g1 >= 0) {
#pragma unroll
        for (int j = 0; j < MPT; ++j) {
          cfma(a2r[j], a2i[j], P2[(g1 % 3) * s2 + m2[j]], C{a1r[j], a1i[j]});
          a1r[j] = a1i[j] = 0;
        }
      }
      g1 = run1;
    }
    if (D == 3 && run2 != g2) {
      if (g2 >= 0) {
#pragma unroll
        for (int j = 0; j < MPT; ++j) {
          cfma(a3r[j], a3i[j], Ph[g2 * nh + m3[j]], C{a2r[j], a2i[j]});
          a2r[j] = a2i[j] = 0;
        }
      }
      g2 = run2;
    }
    const C *ph = phi + (int64_t)g.slot * slot_size + base;
    C v[MPT];
#pragma unroll
    for (int j = 0; j < MPT; ++j) v[j] = ok[j] ? ph[(int64_t)j * blockDim.x] : C{0, 0};
#pragma unroll
    for (int j = 0; j < MPT; ++j) cfma(a1r[j], a1i[j], Pf[(g.code % 3) * n1 + m1[j]], v[j]);
  }
  C *out = psi + (int64_t)dst[i] * slot_size + base;
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    if (g1 >= 0) cfma(a2r[j], a2i[j], P2[(g1 % 3) * s2 + m2[j]], C{a1r[j], a1i[j]});
    if (D == 3) {
      if (g2 >= 0) cfma(a3r[j], a3i[j], Ph[g2 * nh + m3[j]], C{a2r[j], a2i[j]});
      C *o = out + (int64_t)j * blockDim.x;
      if (psi_pitch > 0)  // padded layout of the tcgen05 evaluation: [m3][m2 < pitch][m1 < pitch]
        o = psi + (int64_t)dst[i] * ((int64_t)nh * psi_pitch * psi_pitch) +
            ((int64_t)m3[j] * psi_pitch + m2[j]) * psi_pitch + m1[j];
      if (ok[j] && FGT_OK_PTR(o)) *o = C{a3r[j], a3i[j]};
    } else {
      if (ok[j] && FGT_OK_PTR(&out[(int64_t)j * blockDim.x])) out[(int64_t)j * blockDim.x] = C{a2r[j], a2i[j]};
    }
  }
}


template <int D, typename R>
__global__ void __launch_bounds__(256) gather_kernel(const int32_t *__restrict__ dst, const int64_t *__restrict__ ptr,
                              const GatherSrc *__restrict__ src, const typename C2T<R>::T *__restrict__ Pf,
                              const typename C2T<R>::T *__restrict__ Ph, const typename C2T<R>::T *__restrict__ phi,
                              typename C2T<R>::T *__restrict__ psi, int n1, int nh, int64_t slot_size,
                              int psi_pitch) {
  gather_body<D, R>(dst, ptr, src, Pf, Ph, phi, psi, n1, nh, slot_size, psi_pitch, blockIdx.x, blockIdx.y);
}

// Separable form of the same gather.  A CTA takes one run of up to W target boxes along x_1
// (fixed x_2, x_3) and 256 consecutive modes.  The phase factors are per axis, so the sum over the
// 3^(d-1) neighbouring lines (o_2, o_3) is taken first, position by position along the run
// (w_i = sum_lines P_2(o_2) P_3(o_3) phi[line][i], each of the W + 2 sources loaded once), and the
// x_1 factor last, as a 3-point stencil over w: 9 (W + 2) + 3 W complex products per run in 3D,
// against 27 + 9 + 3 per target for gather_kernel.  The default in every precision (W = 4 when the
// cutoff level has at most 4 boxes a side); FP64 plans built with FGT_GATHER2=0 keep gather_kernel.
template <int D, typename R, int W>
__device__ __forceinline__ void gather2_body(const GatherSeg *__restrict__ segs,
                                                      const typename C2T<R>::T *__restrict__ Pf,
                                                      const typename C2T<R>::T *__restrict__ Ph,
                                                      const typename C2T<R>::T *__restrict__ phi,
                                                      typename C2T<R>::T *__restrict__ psi, int n1, int nh,
                                                      int64_t slot_size, int psi_pitch, int bx, int by) {
  using C = typename C2T<R>::T;
  static_assert(W <= kSegW, "run longer than a GatherSeg");
  constexpr int NL = (D == 3) ? 9 : 3;
  __shared__ GatherSeg sg;
  {
    const int32_t *g = reinterpret_cast<const int32_t *>(segs + bx);
    int32_t *sd = reinterpret_cast<int32_t *>(&sg);
    for (int e = threadIdx.x; e < (int)(sizeof(GatherSeg) / sizeof(int32_t)); e += blockDim.x) sd[e] = g[e];
  }
  __syncthreads();
  const int64_t idx = (int64_t)by * blockDim.x + threadIdx.x;
  if (idx >= slot_size) return;
  int m1, m2, m3;
  mode_index<D>(idx, n1, m1, m2, m3);
  C py[3], pz[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    py[o] = (D == 3) ? Pf[o * n1 + m2] : Ph[o * nh + m2];
    pz[o] = (D == 3) ? Ph[o * nh + m3] : C{1, 0};
  }
  R wr[W + 2], wi[W + 2];
#pragma unroll
  for (int i = 0; i < W + 2; ++i) wr[i] = wi[i] = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int32_t *sl = sg.src[l];
    bool any = false;
#pragma unroll
    for (int i = 0; i < W + 2; ++i) any = any || sl[i] >= 0;
    if (!any) continue;
    C v[W + 2];
#pragma unroll
    for (int i = 0; i < W + 2; ++i) v[i] = (sl[i] >= 0) ? phi[(int64_t)sl[i] * slot_size + idx] : C{0, 0};
    const C f = cmul(py[l % 3], pz[l / 3]);
#pragma unroll
    for (int i = 0; i < W + 2; ++i) cfma(wr[i], wi[i], f, v[i]);
  }
  C px[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) px[o] = Pf[o * n1 + m1];
#pragma unroll
  for (int t = 0; t < W; ++t) {
    if (sg.tgt[t] < 0) continue;
    // source x0 - 1 + i seen from target x0 + t has o_1 = i - 1 - t
    R ar = 0, ai = 0;
    cfma(ar, ai, px[0], C{wr[t], wi[t]});
    cfma(ar, ai, px[1], C{wr[t + 1], wi[t + 1]});
    cfma(ar, ai, px[2], C{wr[t + 2], wi[t + 2]});
    // padded layout of the tcgen05 evaluation when psi_pitch > 0 (3D): [m3][m2 < pitch][m1 < pitch]
    C *o = (D == 3 && psi_pitch > 0)
               ? psi + (int64_t)sg.tgt[t] * ((int64_t)nh * psi_pitch * psi_pitch) +
                     ((int64_t)m3 * psi_pitch + m2) * psi_pitch + m1
               : psi + (int64_t)sg.tgt[t] * slot_size + idx;
    if (FGT_OK_PTR(o)) *o = C{ar, ai};
  }
}


template <int D, typename R, int W>
__global__ void __launch_bounds__(256) gather2_kernel(const GatherSeg *__restrict__ segs,
                                                      const typename C2T<R>::T *__restrict__ Pf,
                                                      const typename C2T<R>::T *__restrict__ Ph,
                                                      const typename C2T<R>::T *__restrict__ phi,
                                                      typename C2T<R>::T *__restrict__ psi, int n1, int nh,
                                                      int64_t slot_size, int psi_pitch) {
  gather2_body<D, R, W>(segs, Pf, Ph, phi, psi, n1, nh, slot_size, psi_pitch, blockIdx.x, blockIdx.y);
}

// The stencil form of the gather over a cutoff grid of NB^3 boxes whether or not every box is an
// anchor (FP64-TC plans, 3D, NB = 4, 8 or 16): MT modes of the grid in shared memory (boxes without an
// outgoing expansion hold zero, which is what the source lists leave out), double-float arithmetic
// in the symmetric form (P(0) = 1, P(+1) = conj P(-1)), each pass a thread per grid line holding the
// line's NB values in registers and writing the stencil back in place.  Every slot is read once
// and written once per mode, where the per-anchor and run forms read each source up to 27 and 9
// times; the price is the stencil over the empty boxes, 3 x 8 double-float products per box.
// Layout: the box slot table, then per mode the boxes with one float4 of padding after each x1 row
// (box b at b + b / NB), so that the x1 lines of consecutive threads fall in different banks.
constexpr int kGridThreads = 512;
template <int NB, int MT>
constexpr size_t gathergrid_smem() {
  return sizeof(int32_t) * NB * NB * NB + sizeof(float4) * (size_t)MT * (NB * NB * NB + NB * NB);
}
template <int NB, int MT>
__global__ void __launch_bounds__(kGridThreads, 1) gathergrid_df_kernel(const int32_t *__restrict__ gslot,
                                                                        const double2 *__restrict__ Pf,
                                                                        const double2 *__restrict__ Ph,
                                                                        const double2 *__restrict__ phi,
                                                                        double2 *__restrict__ psi, int n1, int nh,
                                                                        int64_t slot_size, int periodic) {
  constexpr int NBOX = NB * NB * NB, NL = NB * NB, PN = NBOX + NL, U = 8;
  static_assert((NBOX * sizeof(int32_t)) % 16 == 0, "the slot table must keep the float4 rows aligned");
  extern __shared__ __align__(16) unsigned char gg_raw[];
  int32_t *sslot = reinterpret_cast<int32_t *>(gg_raw);
  float4 *gbuf = reinterpret_cast<float4 *>(gg_raw + sizeof(int32_t) * NBOX);  // [MT][PN]
  for (int b = threadIdx.x; b < NBOX; b += blockDim.x) sslot[b] = __ldg(gslot + b);
  __syncthreads();
  const int64_t m0 = (int64_t)blockIdx.x * MT;
  // MT consecutive modes of a box together; U independent loads in flight per thread
  for (int e0 = threadIdx.x; e0 < MT * NBOX; e0 += U * blockDim.x) {
    double2 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      x[u] = make_double2(0.0, 0.0);
      if (e < MT * NBOX) {
        const int j = e % MT, b = e / MT, sl = sslot[b];
        if (sl >= 0 && m0 + j < slot_size) x[u] = phi[(int64_t)sl * slot_size + m0 + j];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < MT * NBOX) {
        const int j = e % MT, b = e / MT;
        const dfl re = dfl_from_f64(x[u].x), im = dfl_from_f64(x[u].y);
        gbuf[j * PN + b + b / NB] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int ax = 0; ax < 3; ++ax) {
    // padded offsets of the line elements: x1 rows NB + 1 apart, x3 planes NL + NB apart
    const int stride = ax == 0 ? 1 : ax == 1 ? NB + 1 : NL + NB;
    for (int L = threadIdx.x; L < MT * NL; L += blockDim.x) {
      const int j = L / NL, l = L - j * NL;
      const int64_t m = m0 + j;
      if (m >= slot_size) continue;
      int m1, m2, m3;
      mode_index<3>(m, n1, m1, m2, m3);
      const double2 p = ax == 0 ? Pf[m1] : ax == 1 ? Pf[m2] : Ph[m3];  // P(-1) of this axis, in flight
      // the line's first element: l numbers the other two coordinates, the lower one fastest
      const int lo = l % NB, hi = l / NB;
      float4 *ln = gbuf + j * PN + (ax == 0 ? l * (NB + 1) : ax == 1 ? hi * (NL + NB) + lo : hi * (NB + 1) + lo);
      float4 v[NB];
#pragma unroll
      for (int x = 0; x < NB; ++x) v[x] = ln[x * stride];
      const dfl qr = dfl_from_f64(p.x), qi = dfl_from_f64(p.y), nqi = dfl_neg(qi);
#pragma unroll
      for (int x = 0; x < NB; ++x) {
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 lf = x > 0 ? v[x - 1] : (periodic ? v[NB - 1] : zero);
        const float4 rt = x < NB - 1 ? v[x + 1] : (periodic ? v[0] : zero);
        const dfl sr = dfl_add(dfl{lf.x, lf.y}, dfl{rt.x, rt.y}), si = dfl_add(dfl{lf.z, lf.w}, dfl{rt.z, rt.w});
        const dfl dr = dfl_add(dfl{lf.x, lf.y}, dfl{-rt.x, -rt.y}), di = dfl_add(dfl{lf.z, lf.w}, dfl{-rt.z, -rt.w});
        const dfl o_r = dfl_fma(nqi, di, dfl_fma(qr, sr, dfl{v[x].x, v[x].y}));
        const dfl o_i = dfl_fma(qi, dr, dfl_fma(qr, si, dfl{v[x].z, v[x].w}));
        ln[x * stride] = make_float4(o_r.hi, o_r.lo, o_i.hi, o_i.lo);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < MT * NBOX; e += blockDim.x) {
    const int j = e % MT, b = e / MT;
    const int64_t m = m0 + j;
    const int sl = sslot[b];
    if (sl < 0 || m >= slot_size) continue;
    const float4 v = gbuf[j * PN + b + b / NB];
    double2 *o = psi + (int64_t)sl * slot_size + m;
    if (FGT_OK_PTR(o)) *o = make_double2(dfl_to_f64(dfl{v.x, v.y}), dfl_to_f64(dfl{v.z, v.w}));
  }
}

// The run form (gather2) for FP64 expansions with double-float products (FP64-TC plans, 3D): the
// phases of each line (o_2, o_3) formed in FP64, every factor and source split into FP32 pairs with
// integer operations, the 9 (W + 2) + 3 W complex products on the FP32 pipes (about 2^-47 each), the
// result rounded back to FP64.  Used where neither stencil form applies (cutoff grids of more than
// 16 boxes a side, or phases without the exact symmetry the line stencil relies on).
template <int W>
__global__ void __launch_bounds__(256) gather2df_kernel(const GatherSeg *__restrict__ segs,
                                                        const double2 *__restrict__ Pf, const double2 *__restrict__ Ph,
                                                        const double2 *__restrict__ phi, double2 *__restrict__ psi,
                                                        int n1, int nh, int64_t slot_size) {
  static_assert(W <= kSegW, "run longer than a GatherSeg");
  __shared__ GatherSeg sg;
  {
    const int32_t *g = reinterpret_cast<const int32_t *>(segs + blockIdx.x);
    int32_t *sd = reinterpret_cast<int32_t *>(&sg);
    for (int e = threadIdx.x; e < (int)(sizeof(GatherSeg) / sizeof(int32_t)); e += blockDim.x) sd[e] = g[e];
  }
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (idx >= slot_size) return;
  int m1, m2, m3;
  mode_index<3>(idx, n1, m1, m2, m3);
  dfl wr[W + 2], wi[W + 2];
#pragma unroll
  for (int i = 0; i < W + 2; ++i) wr[i] = wi[i] = dfl{0.f, 0.f};
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int32_t *sl = sg.src[l];
    bool any = false;
#pragma unroll
    for (int i = 0; i < W + 2; ++i) any = any || sl[i] >= 0;
    if (!any) continue;
    double2 f;
    {
      const double2 py = Pf[(l % 3) * n1 + m2], pz = Ph[(l / 3) * nh + m3];
      f = make_double2(py.x * pz.x - py.y * pz.y, py.x * pz.y + py.y * pz.x);
    }
    const dfl fr = dfl_from_f64(f.x), fi = dfl_from_f64(f.y), nfi = dfl_neg(fi);
#pragma unroll
    for (int i = 0; i < W + 2; ++i) {
      if (sl[i] < 0) continue;
      const double2 v = phi[(int64_t)sl[i] * slot_size + idx];
      const dfl vr = dfl_from_f64(v.x), vi = dfl_from_f64(v.y);
      wr[i] = dfl_fma(nfi, vi, dfl_fma(fr, vr, wr[i]));
      wi[i] = dfl_fma(fi, vr, dfl_fma(fr, vi, wi[i]));
    }
  }
  dfl pxr[3], pxi[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const double2 p = Pf[o * n1 + m1];
    pxr[o] = dfl_from_f64(p.x);
    pxi[o] = dfl_from_f64(p.y);
  }
#pragma unroll
  for (int t = 0; t < W; ++t) {
    if (sg.tgt[t] < 0) continue;
    dfl ar{0.f, 0.f}, ai{0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 3; ++o) {  // source x0 - 1 + t + o seen from target x0 + t
      ar = dfl_fma(dfl_neg(pxi[o]), wi[t + o], dfl_fma(pxr[o], wr[t + o], ar));
      ai = dfl_fma(pxi[o], wr[t + o], dfl_fma(pxr[o], wi[t + o], ai));
    }
    double2 *op = psi + (int64_t)sg.tgt[t] * slot_size + idx;
    if (FGT_OK_PTR(op)) *op = make_double2(dfl_to_f64(ar), dfl_to_f64(ai));
  }
}

// The same gather for FP64 expansions when every box of the cutoff level is an anchor (3D, NB = 4
// or 8 boxes a side): the phase is a product of one factor per axis and the sources of a target are
// its 3^3 neighbours on the grid, so the sum is a separable 3-point stencil per mode, applied axis by
// axis -- 3 + 3 + 3 complex products per mode and box instead of 27 + 9 + 3 (gather_kernel) or about
// 16 (gather2).  A CTA holds MT consecutive modes of the whole grid in shared memory (ping-pong
// buffers), loads them once (MT contiguous values a slot), runs the three passes (neighbours wrapped
// when periodic, absent in free space) and writes psi once; each thread keeps one mode's nine phase
// factors.  DF (the FP64-TC plans): the products in double-float arithmetic on the FP32 pipes
// (about 2^-47 per operation, far inside the FP64 tolerances), the expansions and phases split into
// FP32 pairs on load and rounded back to FP64 on store with integer operations; otherwise FP64
// arithmetic (FP64-pipe bound).
template <int NB, int MT, bool DF>
__global__ void __launch_bounds__(256) gather3_kernel(const int32_t *__restrict__ gslot, const double2 *__restrict__ Pf,
                                                      const double2 *__restrict__ Ph, const double2 *__restrict__ phi,
                                                      double2 *__restrict__ psi, int n1, int nh, int64_t slot_size,
                                                      int periodic, int sym) {
  static_assert(256 % MT == 0, "modes per CTA must divide the block");
  constexpr int NBOX = NB * NB * NB, BSTEP = 256 / MT;
  extern __shared__ __align__(16) unsigned char g3_raw[];
  // [2][NBOX][MT]: DF (re.hi, re.lo, im.hi, im.lo) as float4, else the double2 itself
  float4 *buf = reinterpret_cast<float4 *>(g3_raw);
  double2 *bufd = reinterpret_cast<double2 *>(g3_raw);
  const int j = threadIdx.x % MT, b0 = threadIdx.x / MT;
  const int64_t m = (int64_t)blockIdx.x * MT + j;
  const bool live = m < slot_size;
  int m1 = 0, m2 = 0, m3 = 0;
  mode_index<3>(live ? m : 0, n1, m1, m2, m3);
  double2 P[3][3];  // [axis][o + 1]
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    P[0][o] = Pf[o * n1 + m1];
    P[1][o] = Pf[o * n1 + m2];
    P[2][o] = Ph[o * nh + m3];
  }
  dfl pr[3][3], pi[3][3];
  if constexpr (DF) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        pr[ax][o] = dfl_from_f64(P[ax][o].x);
        pi[ax][o] = dfl_from_f64(P[ax][o].y);
      }
  }
  for (int b = b0; b < NBOX; b += BSTEP) {
    const double2 x = live ? phi[(int64_t)__ldg(gslot + b) * slot_size + m] : make_double2(0.0, 0.0);
    if constexpr (DF) {
      const dfl re = dfl_from_f64(x.x), im = dfl_from_f64(x.y);
      buf[b * MT + j] = make_float4(re.hi, re.lo, im.hi, im.lo);
    } else {
      bufd[b * MT + j] = x;
    }
  }
  __syncthreads();
  int cur = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int stride = ax == 0 ? 1 : ax == 1 ? NB : NB * NB;
    const int ib = cur * NBOX * MT, ob = (1 - cur) * NBOX * MT;
    for (int b = b0; b < NBOX; b += BSTEP) {
      const int x = (b / stride) % NB;
      if constexpr (DF) {
        if (sym) {
          // P(0) = 1 and P(+1) = conj P(-1) = (pr, -pi): P(-1) l + P(+1) r = pr (l + r) + i pi (l - r),
          // 4 double-float products instead of 12
          const int xl = x - 1, xr = x + 1;
          float4 l = make_float4(0.f, 0.f, 0.f, 0.f), r = l;
          if (xl >= 0 || periodic) l = buf[ib + (b + (((xl + NB) % NB) - x) * stride) * MT + j];
          if (xr < NB || periodic) r = buf[ib + (b + (((xr + NB) % NB) - x) * stride) * MT + j];
          const float4 c = buf[ib + b * MT + j];
          const dfl sr = dfl_add(dfl{l.x, l.y}, dfl{r.x, r.y}), si = dfl_add(dfl{l.z, l.w}, dfl{r.z, r.w});
          const dfl dr_ = dfl_add(dfl{l.x, l.y}, dfl_neg(dfl{r.x, r.y}));
          const dfl di_ = dfl_add(dfl{l.z, l.w}, dfl_neg(dfl{r.z, r.w}));
          const dfl qr = pr[ax][0], qi = pi[ax][0];
          const dfl orr = dfl_fma(dfl_neg(qi), di_, dfl_fma(qr, sr, dfl{c.x, c.y}));
          const dfl oii = dfl_fma(qi, dr_, dfl_fma(qr, si, dfl{c.z, c.w}));
          buf[ob + b * MT + j] = make_float4(orr.hi, orr.lo, oii.hi, oii.lo);
          continue;
        }
      }
      dfl ar{0.f, 0.f}, ai{0.f, 0.f};
      double dr = 0.0, di = 0.0;
#pragma unroll
      for (int o = -1; o <= 1; ++o) {
        int xs = x + o;
        if (xs < 0 || xs >= NB) {
          if (!periodic) continue;
          xs = (xs + NB) % NB;
        }
        const int src = ib + (b + (xs - x) * stride) * MT + j;
        if constexpr (DF) {
          const float4 v = buf[src];
          const dfl vr{v.x, v.y}, vi{v.z, v.w}, qr = pr[ax][o + 1], qi = pi[ax][o + 1];
          const dfl nqi{-qi.hi, -qi.lo};
          ar = dfl_fma(qr, vr, ar);  // (qr + i qi)(vr + i vi)
          ar = dfl_fma(nqi, vi, ar);
          ai = dfl_fma(qr, vi, ai);
          ai = dfl_fma(qi, vr, ai);
        } else {
          cfma(dr, di, P[ax][o + 1], bufd[src]);
        }
      }
      if constexpr (DF) buf[ob + b * MT + j] = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
      else bufd[ob + b * MT + j] = make_double2(dr, di);
    }
    __syncthreads();
    cur = 1 - cur;
  }
  if (!live) return;
  for (int b = b0; b < NBOX; b += BSTEP) {
    const int src = cur * NBOX * MT + b * MT + j;
    double2 *o = psi + (int64_t)__ldg(gslot + b) * slot_size + m;
    double2 r;
    if constexpr (DF) {
      const float4 v = buf[src];
      r = make_double2(dfl_to_f64(dfl{v.x, v.y}), dfl_to_f64(dfl{v.z, v.w}));
    } else {
      r = bufd[src];
    }
    if (FGT_OK_PTR(o)) *o = r;
  }
}

constexpr int gather3_mt(int nb) { return nb == 4 ? 16 : 4; }

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
  // the phase is a product of one factor per axis, so the 2^d children are combined axis by axis:
  // pairs along x_1, then along x_2, then along the last (half-range) axis -- 14 complex products
  // per mode in 3D instead of 8 phase builds (16 products) and 8 applications
  const C q10 = qf[m1], q11 = qf[n1 + m1];
  const int ml = (D == 3) ? m3 : m2;  // last axis: half range
  const C ql0 = qh[ml], ql1 = qh[nh + ml];
  C w[2];
#pragma unroll
  for (int bl = 0; bl < 2; ++bl) {          // last-axis half (child bit d - 1)
    R sr = 0, si = 0;
#pragma unroll
    for (int b2 = 0; b2 < (D == 3 ? 2 : 1); ++b2) {
      const int c0 = (D == 3) ? ((b2 << 1) | (bl << 2)) : (bl << 1);
      R tr = 0, ti = 0;                      // x_1 pair (child bit 0)
      cfma(tr, ti, q10, phi[(int64_t)it.child[c0] * slot_size + idx]);
      cfma(tr, ti, q11, phi[(int64_t)it.child[c0 | 1] * slot_size + idx]);
      if (D == 3) cfma(sr, si, qf[b2 * n1 + m2], C{tr, ti});  // x_2 pair (child bit 1)
      else { sr = tr; si = ti; }
    }
    w[bl] = C{sr, si};
  }
  R ar = 0, ai = 0;
  cfma(ar, ai, ql0, w[0]);
  cfma(ar, ai, ql1, w[1]);
  if (FGT_OK_PTR(&phi[(int64_t)it.parent * slot_size + idx])) phi[(int64_t)it.parent * slot_size + idx] = C{ar, ai};
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
  // the phase axis by axis: the last (half-range) axis, then x_2, then x_1 -- 14 complex products
  // per mode in 3D instead of 8 phase builds and 8 applications
  const int ml = (D == 3) ? m3 : m2;
  const C q10 = qf[m1], q11 = qf[n1 + m1];
#pragma unroll
  for (int bl = 0; bl < 2; ++bl) {
    const C wl = cmul(qh[bl * nh + ml], v);
#pragma unroll
    for (int b2 = 0; b2 < (D == 3 ? 2 : 1); ++b2) {
      const C w2 = (D == 3) ? cmul(qf[b2 * n1 + m2], wl) : wl;
      const int c0 = (D == 3) ? ((b2 << 1) | (bl << 2)) : (bl << 1);
      C *o0 = &psi[(int64_t)it.child[c0] * slot_size + idx], *o1 = &psi[(int64_t)it.child[c0 | 1] * slot_size + idx];
      if (FGT_OK_PTR(o0)) *o0 = cmul(q10, w2);
      if (FGT_OK_PTR(o1)) *o1 = cmul(q11, w2);
    }
  }
}

// ----------------------------------------------------------------------------- near field

// One D-list pair per CTA: u_T += (K_d x ... x K_1) sigma_S with the three k x k tables of the
// pair, added to u with FP64 atomics (u is cleared before the evaluation step stores into it).
// Pair-parallel so that many pairs are in flight at once; the tables, their row bands and sigma_S
// are staged in shared memory.  Each row of a table is applied over its band only (the columns
// whose entries matter): the full row for wide Gaussians, a few columns as delta -> 0.
template <int D>
__device__ __forceinline__ void near2_body(const NearPair *__restrict__ pairs, const double *__restrict__ tab,
                                                    const int16_t *__restrict__ band,
                                                    const double *__restrict__ sigma, double *__restrict__ u, int k, int bx, int by) {
  extern __shared__ double sm[];
  const int kk = k * k;
  const int np = (D == 3) ? kk * k : kk;
  double *s0 = sm, *A = sm + np, *B = A + np, *T = B + np;
  int16_t *bd = reinterpret_cast<int16_t *>(T + D * kk);  // [D][k][2]
  const NearPair pr = pairs[bx];
  const double *sg = sigma + pr.src * np;
  for (int e = threadIdx.x; e < np; e += blockDim.x) s0[e] = FGT_OK_PTR(sg + e) ? __ldg(sg + e) : 0.0;
  for (int e = threadIdx.x; e < D * kk; e += blockDim.x) {
    const int a = e / kk;
    T[e] = __ldg(tab + (int64_t)pr.tab[a] * kk + (e - a * kk));
  }
  for (int e = threadIdx.x; e < D * 2 * k; e += blockDim.x) {
    const int a = e / (2 * k);
    bd[e] = __ldg(band + (int64_t)pr.tab[a] * 2 * k + (e - a * 2 * k));
  }
  __syncthreads();
  double *ut = u + pr.tgt * np;
  if (D == 3) {
    for (int e = threadIdx.x; e < np; e += blockDim.x) {  // A[j3][j2][t1] = sum_j1 T1[t1][j1] s0[j3][j2][j1]
      const int row = e / k, t1 = e - row * k;
      const double *sp = s0 + row * k, *tp = T + t1 * k;
      double a = 0;
      for (int j = bd[2 * t1]; j <= bd[2 * t1 + 1]; ++j) a = fma(tp[j], sp[j], a);
      A[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np; e += blockDim.x) {  // B[j3][t2][t1] = sum_j2 T2[t2][j2] A[j3][j2][t1]
      const int j3 = e / kk, rem = e - j3 * kk, t2 = rem / k, t1 = rem - t2 * k;
      const double *tp = T + kk + t2 * k, *ap = A + j3 * kk + t1;
      const int16_t *b2 = bd + 2 * k + 2 * t2;
      double a = 0;
      for (int j = b2[0]; j <= b2[1]; ++j) a = fma(tp[j], ap[j * k], a);
      B[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np; e += blockDim.x) {  // u[t3][t2][t1] += sum_j3 T3[t3][j3] B[j3][t2][t1]
      const int t3 = e / kk, rem = e - t3 * kk;
      const double *tp = T + 2 * kk + t3 * k, *bp = B + rem;
      const int16_t *b3 = bd + 4 * k + 2 * t3;
      if (b3[1] < b3[0]) continue;
      double a = 0;
      for (int j = b3[0]; j <= b3[1]; ++j) a = fma(tp[j], bp[j * kk], a);
      if (FGT_OK_PTR(ut + e)) atomicAdd(ut + e, a);
    }
  } else {
    for (int e = threadIdx.x; e < np; e += blockDim.x) {  // A[j2][t1] = sum_j1 T1[t1][j1] s0[j2][j1]
      const int j2 = e / k, t1 = e - j2 * k;
      const double *sp = s0 + j2 * k, *tp = T + t1 * k;
      double a = 0;
      for (int j = bd[2 * t1]; j <= bd[2 * t1 + 1]; ++j) a = fma(tp[j], sp[j], a);
      A[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < np; e += blockDim.x) {  // u[t2][t1] += sum_j2 T2[t2][j2] A[j2][t1]
      const int t2 = e / k, t1 = e - t2 * k;
      const double *tp = T + kk + t2 * k, *ap = A + t1;
      const int16_t *b2 = bd + 2 * k + 2 * t2;
      if (b2[1] < b2[0]) continue;
      double a = 0;
      for (int j = b2[0]; j <= b2[1]; ++j) a = fma(tp[j], ap[j * k], a);
      if (FGT_OK_PTR(ut + e)) atomicAdd(ut + e, a);
    }
  }
}


// The same 3D near field with double-float products (FP64-TC plans): σ and the three tables split
// into FP32 pairs on load (integer operations), the three passes on the FP32 pipes (about 2^-47 a
// product), each result rounded back to FP64 for the atomic addition into u.
__global__ void __launch_bounds__(128) near2df_kernel(const NearPair *__restrict__ pairs,
                                                      const double *__restrict__ tab,
                                                      const int16_t *__restrict__ band,
                                                      const double *__restrict__ sigma, double *__restrict__ u, int k) {
  extern __shared__ float2 smf[];
  const int kk = k * k, np = kk * k;
  float2 *s0 = smf, *A = smf + np, *B = A + np, *T = B + np;
  int16_t *bd = reinterpret_cast<int16_t *>(T + 3 * kk);  // [3][k][2]
  const NearPair pr = pairs[blockIdx.x];
  const double *sg = sigma + pr.src * np;
  auto put = [](float2 *p, double x) {
    const dfl v = dfl_from_f64(x);
    *p = make_float2(v.hi, v.lo);
  };
  for (int e = threadIdx.x; e < np; e += blockDim.x) put(s0 + e, FGT_OK_PTR(sg + e) ? __ldg(sg + e) : 0.0);
  for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
    const int a = e / kk;
    put(T + e, __ldg(tab + (int64_t)pr.tab[a] * kk + (e - a * kk)));
  }
  for (int e = threadIdx.x; e < 3 * 2 * k; e += blockDim.x) {
    const int a = e / (2 * k);
    bd[e] = __ldg(band + (int64_t)pr.tab[a] * 2 * k + (e - a * 2 * k));
  }
  __syncthreads();
  auto ld = [](const float2 *p) { const float2 v = *p; return dfl{v.x, v.y}; };
  for (int e = threadIdx.x; e < np; e += blockDim.x) {  // A[j3][j2][t1] = sum_j1 T1[t1][j1] s0[j3][j2][j1]
    const int row = e / k, t1 = e - row * k;
    const float2 *sp = s0 + row * k, *tp = T + t1 * k;
    dfl a{0.f, 0.f};
    for (int j = bd[2 * t1]; j <= bd[2 * t1 + 1]; ++j) a = dfl_fma(ld(tp + j), ld(sp + j), a);
    A[e] = make_float2(a.hi, a.lo);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < np; e += blockDim.x) {  // B[j3][t2][t1] = sum_j2 T2[t2][j2] A[j3][j2][t1]
    const int j3 = e / kk, rem = e - j3 * kk, t2 = rem / k, t1 = rem - t2 * k;
    const float2 *tp = T + kk + t2 * k, *ap = A + j3 * kk + t1;
    const int16_t *b2 = bd + 2 * k + 2 * t2;
    dfl a{0.f, 0.f};
    for (int j = b2[0]; j <= b2[1]; ++j) a = dfl_fma(ld(tp + j), ld(ap + j * k), a);
    B[e] = make_float2(a.hi, a.lo);
  }
  __syncthreads();
  double *ut = u + pr.tgt * np;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {  // u[t3][t2][t1] += sum_j3 T3[t3][j3] B[j3][t2][t1]
    const int t3 = e / kk, rem = e - t3 * kk;
    const float2 *tp = T + 2 * kk + t3 * k, *bp = B + rem;
    const int16_t *b3 = bd + 4 * k + 2 * t3;
    if (b3[1] < b3[0]) continue;
    dfl a{0.f, 0.f};
    for (int j = b3[0]; j <= b3[1]; ++j) a = dfl_fma(ld(tp + j), ld(bp + j * kk), a);
    if (FGT_OK_PTR(ut + e)) atomicAdd(ut + e, dfl_to_f64(a));
  }
}

template <int D>
__global__ void __launch_bounds__(128) near2_kernel(const NearPair *__restrict__ pairs, const double *__restrict__ tab,
                                                    const int16_t *__restrict__ band,
                                                    const double *__restrict__ sigma, double *__restrict__ u, int k) {
  near2_body<D>(pairs, tab, band, sigma, u, k, blockIdx.x, blockIdx.y);
}

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
    for (int e = threadIdx.x; e < np; e += blockDim.x) s0[e] = FGT_OK_PTR(sg + e) ? __ldg(sg + e) : 0.0;
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

// The second and later launches of a phase go to side streams 1.. (round robin), forked from the
// caller's stream before the first of them and joined back into it at the end of the phase, so
// per-size launches with few CTAs (large blocks) run beside the others instead of after them.
struct Spread {
  const ExecDesc &e;
  cudaStream_t st;
  int n = 0;
  bool used[kSides] = {};
  cudaError_t err = cudaSuccess;
  // the fork point is the construction: side launches wait for what st holds now, not for the
  // phase's own first launch
  Spread(const ExecDesc &ex, cudaStream_t s) : e(ex), st(s) {
    if (e.side[1] != nullptr) err = cudaEventRecord(e.fork_ev[1], st);
  }
  cudaStream_t next() {
    const int j = n++;
    if (j == 0 || e.side[1] == nullptr) return st;
    const int sd = 1 + (j - 1) % (kSides - 1);
    if (!used[sd]) {
      cudaError_t r = cudaStreamWaitEvent(e.side[sd], e.fork_ev[1], 0);
      if (r != cudaSuccess && err == cudaSuccess) err = r;
      used[sd] = true;
    }
    return e.side[sd];
  }
  cudaError_t join() {
    for (int sd = 1; sd < kSides; ++sd) {
      if (!used[sd]) continue;
      cudaError_t r = cudaEventRecord(e.join_ev[sd], e.side[sd]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, e.join_ev[sd], 0);
      if (r != cudaSuccess && err == cudaSuccess) err = r;
      used[sd] = false;
    }
    n = 0;
    return err;
  }
};

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
  if (e.zero_u) {
    // the near field (and the evaluation of cutoff-level leaves) add into u: clear it first
    if ((err = cudaMemsetAsync(u, 0, sizeof(double) * (size_t)e.n_points, st)) != cudaSuccess) return err;
  }
  // near field: D-list pairs, FP64; independent of the plane-wave phases, so it runs on the
  // plan's second stream (forked after the clear of u, joined before returning) when one exists
  auto launch_near = [&](cudaStream_t ns) -> cudaError_t {
    const int np = D == 3 ? e.k * e.k * e.k : e.k * e.k;
    const size_t nsm = sizeof(double) * (3 * (size_t)np + (size_t)D * e.k * e.k) + sizeof(int16_t) * 2 * D * e.k;
    // FP64-TC plans in 3D: the near field's products in double-float arithmetic (same shared memory)
    const bool df = D == 3 && e.tc64 != 0;
    cudaError_t r = df ? cudaFuncSetAttribute(near2df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm)
                       : cudaFuncSetAttribute(near2_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm);
    if (r != cudaSuccess) return r;
    if (e.events) cudaEventRecord(e.events[10], ns);
    if (df)
      near2df_kernel<<<(unsigned)e.n_near_pairs, 128, nsm, ns>>>(e.near_pairs, e.near_tab, e.near_band, sigma, u, e.k);
    else
      near2_kernel<D><<<(unsigned)e.n_near_pairs, 128, nsm, ns>>>(e.near_pairs, e.near_tab, e.near_band, sigma, u, e.k);
    r = cudaGetLastError();
    if (e.events) cudaEventRecord(e.events[11], ns);
    return r;
  };
  const bool near_aside = e.n_near_pairs > 0 && e.side[0] != nullptr;
  if (!(e.n_near_pairs > 0) && e.events) {
    cudaEventRecord(e.events[10], st);
    cudaEventRecord(e.events[11], st);
  }
  auto fork_near = [&](int phase) -> cudaError_t {
    if (!near_aside || e.near_phase != phase) return cudaSuccess;
    cudaError_t r;
    if ((r = cudaEventRecord(e.fork_ev[0], st)) != cudaSuccess) return r;
    if ((r = cudaStreamWaitEvent(e.side[0], e.fork_ev[0], 0)) != cudaSuccess) return r;
    if ((r = launch_near(e.side[0])) != cudaSuccess) return r;
    return cudaEventRecord(e.join_ev[0], e.side[0]);
  };
  if ((err = fork_near(0)) != cudaSuccess) return err;
  if (e.n_blocks > 0) {
    // outgoing expansions: zero, then every block adds its contribution (unless every block is the
    // only one of its anchor and stores the whole slot)
    // FP64 on the BF16 tensor cores by exact slicing: three contraction stages through the scratch
    // arrays (their absence -- the allocation-free call -- leaves the FP64 kernels below)
    const bool oz_form = D == 3 && sizeof(R) == 8 && e.oz && e.oz_x != nullptr;
    if (!(oz_form ? e.oz_sole : e.phi_stored) &&
        (err = cudaMemsetAsync(phi, 0, sizeof(C) * ss * e.n_phi_slots, st)) != cudaSuccess)
      return err;
    if (oz_form) {
      if ((err = run_oz_stage(e, 0, sigma, e.oz_x, st)) != cudaSuccess) return err;
      if ((err = run_oz_stage(e, 1, e.oz_x, e.oz_y, st)) != cudaSuccess) return err;
      if ((err = run_oz_stage(e, 2, e.oz_y, reinterpret_cast<double *>(phi), st)) != cudaSuccess) return err;
    } else {
    if (D == 3 && sizeof(R) == 4 && e.sigp != nullptr && e.n_pack > 0) {
      sigma_pack_kernel<<<(unsigned)e.n_pack, 256, 0, st>>>(e.blocks, e.pack_block, e.block_leaves, sigma, e.sigp,
                                                            e.k);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    Spread fs(e, st);
    if (e.n_f1 > 0) {
      const size_t fsm = form_smem_bytes(D, e.Kmax_f1, n1, sizeof(R) == 4);
      if ((err = cudaFuncSetAttribute(form_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm)) !=
          cudaSuccess)
        return err;
      form_kernel<D, R><<<dim3((unsigned)e.n_f1, (unsigned)nh), 256, fsm, fs.next()>>>(
          e.f1_blocks, e.block_leaves, sigma, reinterpret_cast<const C *>(e.Ff), reinterpret_cast<const C *>(e.Fh),
          phi, e.k, n1, nh, ss, e.Kmax_f1);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    for (const LaunchRange &lr : e.f2_ranges) {  // one launch per block size K
      if (D == 3 && lr.tensor == 7 && sizeof(R) == 4 &&
          (e.sig_order != 1 || e.sigp == nullptr || !e.sig_maps_ready)) {
        // without the packed density in its order (the allocation-free call): the register-tiled
        // tensor-core form, one block per CTA, reading sigma itself, adding into the cleared slot
        const bool big = lr.K > 16, small_n = n1_pad8(n1) / 4 <= 8;
        auto fk = big ? (small_n ? form4_kernel<8, true> : form4_kernel<kNbtMax, true>)
                      : (small_n ? form4_kernel<8, false> : form4_kernel<kNbtMax, false>);
        const size_t fsm = big ? form4b_bytes(lr.K, n1) : form4_bytes(1, lr.K, n1);
        if ((err = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm)) != cudaSuccess)
          return err;
        fk<<<(unsigned)(lr.count * ((nh + kSc - 1) / kSc)), 256, fsm, fs.next()>>>(
            e.f2_blocks, e.f2_gptr + lr.first, e.block_leaves, sigma, nullptr, reinterpret_cast<const float2 *>(e.Ff),
            reinterpret_cast<const float2 *>(e.Fh), reinterpret_cast<float2 *>(phi), e.k, n1, nh, ss);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        continue;
      }
      if (D == 3 && lr.tensor == 7 && sizeof(R) == 4) {  // all stages on tcgen05
        const int ki = lr.K == 8 ? 0 : lr.K == 16 ? 1 : 2;
        auto k7 = ki == 0 ? form7_kernel<8, 16> : ki == 1 ? form7_kernel<16, 16> : form7_kernel<32, 16>;
        if ((err = cudaFuncSetAttribute(k7, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) !=
            cudaSuccess)
          return err;
        k7<<<(unsigned)lr.count, 512, lr.smem, fs.next()>>>(
            e.sig_map[ki], e.f2_blocks + lr.first, reinterpret_cast<const float2 *>(e.Ff),
            reinterpret_cast<const float2 *>(e.Fh), reinterpret_cast<float2 *>(phi), e.k, n1, nh, ss);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        continue;
      }
      if (D == 3 && lr.tensor == 7) return cudaErrorNotSupported;  // needs the packed density
      if (D == 3 && lr.tensor && sizeof(R) == 4) {
        const bool small_n = n1_pad8(n1) / 4 <= 8;
        auto fk = lr.big ? (small_n ? form4_kernel<8, true> : form4_kernel<kNbtMax, true>)
                         : (small_n ? form4_kernel<8, false> : form4_kernel<kNbtMax, false>);
        if ((err = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) !=
            cudaSuccess)
          return err;
        fk<<<(unsigned)(lr.count * ((nh + kSc - 1) / kSc)), 256, lr.smem, fs.next()>>>(
            e.f2_blocks, e.f2_gptr + lr.first, e.block_leaves, sigma, e.sigp, reinterpret_cast<const float2 *>(e.Ff),
            reinterpret_cast<const float2 *>(e.Fh), reinterpret_cast<float2 *>(phi), e.k, n1, nh, ss);
      } else if (D == 3) {
        auto f3 = lr.tensor ? form3_kernel<R, true> : form3_kernel<R, false>;
        if ((err = cudaFuncSetAttribute(f3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) !=
            cudaSuccess)
          return err;
        f3<<<dim3((unsigned)lr.count, (unsigned)((nh + kSc - 1) / kSc)), 256, lr.smem, fs.next()>>>(
            e.f2_blocks, e.f2_gptr + lr.first, e.block_leaves, sigma, reinterpret_cast<const C *>(e.Ff),
            reinterpret_cast<const C *>(e.Fh), phi, e.k, n1, nh, ss);
      } else {
        if ((err = cudaFuncSetAttribute(form2_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)lr.smem)) != cudaSuccess)
          return err;
        form2_kernel<D, R><<<dim3((unsigned)lr.count, (unsigned)nh), 256, lr.smem, fs.next()>>>(
            e.f2_blocks, e.f2_gptr + lr.first, e.block_leaves, sigma, reinterpret_cast<const C *>(e.Ff),
            reinterpret_cast<const C *>(e.Fh), phi, e.k, n1, nh, ss);
      }
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if ((err = fs.join()) != cudaSuccess) return err;
    }
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
  if ((err = fork_near(2)) != cudaSuccess) return err;
  mark(2, 0);
  const C *eval_src = phi;
  if (!e.fourier && e.n_gather > 0) {
    if (D == 3 && sizeof(R) == 8 && e.tc64 && e.grid_lines && e.gather_sym && e.gather_grid != nullptr &&
        e.psi_pitch == 0 && (e.grid_nb == 4 || e.grid_nb == 8 || e.grid_nb == 16)) {
      // FP64-TC: the in-place line stencil over the whole grid (empty boxes as zero)
      const int nb = e.grid_nb, mt = nb == 4 ? 176 : nb == 8 ? 24 : 3;
      auto gk = nb == 4 ? gathergrid_df_kernel<4, 176> : nb == 8 ? gathergrid_df_kernel<8, 24>
                                                                 : gathergrid_df_kernel<16, 3>;
      const size_t gsm = nb == 4 ? gathergrid_smem<4, 176>() : nb == 8 ? gathergrid_smem<8, 24>()
                                                                       : gathergrid_smem<16, 3>();
      if ((err = cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)) != cudaSuccess)
        return err;
      gk<<<(unsigned)((ss + mt - 1) / mt), kGridThreads, gsm, st>>>(
          e.gather_grid, reinterpret_cast<const double2 *>(e.Pf), reinterpret_cast<const double2 *>(e.Ph),
          reinterpret_cast<const double2 *>(phi), reinterpret_cast<double2 *>(psi), n1, nh, ss, e.grid_periodic);
    } else if (D == 3 && sizeof(R) == 8 && (e.grid_nb == 4 || e.grid_nb == 8) && !e.grid_lines &&
               e.gather_grid != nullptr && e.psi_pitch == 0) {
      // FP64, every box of the cutoff level an anchor: the stencil form, axis by axis
      const int nb = e.grid_nb, mt = gather3_mt(nb);
      // FP64-TC plans: double-float products; FP64 plans: FP64 products
      auto g3 = e.tc64 ? (nb == 4 ? gather3_kernel<4, gather3_mt(4), true> : gather3_kernel<8, gather3_mt(8), true>)
                       : (nb == 4 ? gather3_kernel<4, gather3_mt(4), false> : gather3_kernel<8, gather3_mt(8), false>);
      const size_t gsm = 2 * sizeof(float4) * (size_t)nb * nb * nb * mt;
      if ((err = cudaFuncSetAttribute(g3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm)) != cudaSuccess)
        return err;
      g3<<<(unsigned)((ss + mt - 1) / mt), 256, gsm, st>>>(
          e.gather_grid, reinterpret_cast<const double2 *>(e.Pf), reinterpret_cast<const double2 *>(e.Ph),
          reinterpret_cast<const double2 *>(phi), reinterpret_cast<double2 *>(psi), n1, nh, ss, e.grid_periodic,
          e.gather_sym);
    } else if (D == 3 && sizeof(R) == 8 && e.tc64 && e.n_gather_segs > 0 && e.psi_pitch == 0) {
      // FP64-TC: the run form with double-float products
      auto g2 = (e.seg_w > 0 && e.seg_w <= 4) ? gather2df_kernel<4> : gather2df_kernel<kSegW>;
      g2<<<dim3((unsigned)e.n_gather_segs, tiles), 256, 0, st>>>(
          e.gather_segs, reinterpret_cast<const double2 *>(e.Pf), reinterpret_cast<const double2 *>(e.Ph),
          reinterpret_cast<const double2 *>(phi), reinterpret_cast<double2 *>(psi), n1, nh, ss);
    } else if (e.n_gather_segs > 0) {
      // runs of at most 4 targets (4 boxes a side at the cutoff level): the 4-wide kernel, which
      // does not spend products on the empty positions of an 8-wide run
      auto g2 = (e.seg_w > 0 && e.seg_w <= 4) ? gather2_kernel<D, R, 4> : gather2_kernel<D, R, kSegW>;
      g2<<<dim3((unsigned)e.n_gather_segs, tiles), 256, 0, st>>>(
          e.gather_segs, reinterpret_cast<const C *>(e.Pf), reinterpret_cast<const C *>(e.Ph), phi, psi, n1, nh, ss,
          e.psi_pitch);
    } else {
      const unsigned gtiles = (unsigned)((ss + 256 * kGatherMpt - 1) / (256 * kGatherMpt));
      gather_kernel<D, R><<<dim3((unsigned)e.n_gather, gtiles), 256, 0, st>>>(
          e.gather_dst, e.gather_ptr, e.gather_src, reinterpret_cast<const C *>(e.Pf),
          reinterpret_cast<const C *>(e.Ph), phi, psi, n1, nh, ss, e.psi_pitch);
    }
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
  if ((err = fork_near(4)) != cudaSuccess) return err;
  mark(4, 0);
  if (D == 3 && sizeof(R) == 4 && e.psi_tc != nullptr && e.n_psi_tc_slots > 0) {
    // the expansions the tcgen05 evaluation reads, in its operand layout (before the fork below)
    const int64_t items = (int64_t)((n1 * n1 + 127) / 128) * (eval6_kpad(nh) / 4) * 128 * e.n_psi_tc_slots;
    const unsigned g = (unsigned)std::min<int64_t>((items + 255) / 256, 152 * 16);
    psi_tc_kernel<<<g, 256, 0, st>>>(reinterpret_cast<const float2 *>(eval_src),
                                     static_cast<unsigned char *>(e.psi_tc), n1, nh, ss, e.n_psi_tc_slots);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const bool oz_eval = D == 3 && sizeof(R) == 8 && e.oz && e.oz_x != nullptr;
  if (oz_eval) {
    if ((err = run_oz_stage(e, 3, reinterpret_cast<const double *>(eval_src), e.oz_x, st)) != cudaSuccess) return err;
    if ((err = run_oz_stage(e, 4, e.oz_x, e.oz_y, st)) != cudaSuccess) return err;
    if ((err = run_oz_stage(e, 5, e.oz_y, u, st)) != cudaSuccess) return err;
  }
  Spread es(e, st);
  if (e.n_e1 > 0 && !oz_eval) {
    const size_t esm = eval_smem_bytes(D, e.Kmax_e1, n1, sizeof(R) == 4);
    if ((err = cudaFuncSetAttribute(eval_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm)) !=
        cudaSuccess)
      return err;
    eval_kernel<D, R><<<dim3((unsigned)e.n_e1, (unsigned)e.Kmax_e1), 256, esm, es.next()>>>(
        e.e1_blocks, e.eval_leaves, reinterpret_cast<const C *>(e.Ef), reinterpret_cast<const C *>(e.Eh), eval_src,
        u, e.k, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  for (const LaunchRange &lr : e.e2_ranges) {  // one launch per block size K
    if (oz_eval) break;
    if (D == 3 && lr.tensor == 7 && sizeof(R) == 4 && e.psi_pitch == e7::kP && e.psi_map_ready) {
      // all stages on tcgen05
      // 16 warps for K = 32 blocks, 8 for the smaller ones (measured: the extra warps hide the latency
      // of the large blocks' phases, and cost more in barriers than they gain on small blocks)
      auto k7 = lr.K == 8 ? eval7_kernel<8, 8> : lr.K == 16 ? eval7_kernel<16, 8> : eval7_kernel<32, 16>;
      const unsigned nt = lr.K == 32 ? 512 : 256;
      if ((err = cudaFuncSetAttribute(k7, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) != cudaSuccess)
        return err;
      k7<<<(unsigned)lr.count, nt, lr.smem, es.next()>>>(e.psi_map, e.e2_blocks + lr.first, e.eval_leaves,
                                                          reinterpret_cast<const float2 *>(e.Ef),
                                                          reinterpret_cast<const float2 *>(e.Eh), u, e.k, n1, nh);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      continue;
    }
    if (D == 3 && lr.tensor == 1 && sizeof(R) == 4) {
      auto tk = (2 * nh <= 32) ? eval3_kernel<4> : eval3_kernel<8>;
      if ((err = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) != cudaSuccess)
        return err;
      tk<<<dim3((unsigned)lr.count, (unsigned)((lr.K + kEvalRows - 1) / kEvalRows)), 256, lr.smem, es.next()>>>(
          e.e2_blocks + lr.first, e.eval_leaves,
                                                   reinterpret_cast<const float2 *>(e.Ef),
                                                   reinterpret_cast<const float2 *>(e.Eh),
                                                   reinterpret_cast<const float2 *>(eval_src), u, e.k, n1, nh, ss);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      continue;
    }
    if (D == 3 && lr.tensor == 4 && sizeof(R) == 4 && e.psi_tc != nullptr) {  // stage 1 on tcgen05
      auto k6 = lr.rows <= 4 ? eval6_kernel<4> : lr.rows <= 8 ? eval6_kernel<8> : eval6_kernel<16>;
      const int rows6 = lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16;
      if ((err = cudaFuncSetAttribute(k6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) != cudaSuccess)
        return err;
      k6<<<dim3((unsigned)lr.count, (unsigned)((lr.K + rows6 - 1) / rows6)), 256, lr.smem, es.next()>>>(
          e.e2_blocks + lr.first, e.eval_leaves, reinterpret_cast<const float2 *>(e.Ef),
          reinterpret_cast<const float2 *>(e.Eh), static_cast<const unsigned char *>(e.psi_tc), u, e.k, n1, nh,
          lr.tmem_cols);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      continue;
    }
    if (D == 3 && lr.tensor == 3) {  // half-range axis contracted last
      auto k5 = lr.rows <= 1   ? eval5_kernel<R, 1>
                : lr.rows <= 2 ? eval5_kernel<R, 2>
                : lr.rows <= 4 ? eval5_kernel<R, 4>
                : lr.rows <= 8 ? eval5_kernel<R, 8>
                               : eval5_kernel<R, 16>;
      const int rc = lr.rows <= 1 ? 1 : lr.rows <= 2 ? 2 : lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16;
      if ((err = cudaFuncSetAttribute(k5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) != cudaSuccess)
        return err;
      k5<<<dim3((unsigned)lr.count, (unsigned)((lr.K + rc - 1) / rc)), 256, lr.smem, es.next()>>>(
          e.e2_blocks + lr.first, e.eval_leaves, reinterpret_cast<const C *>(e.Ef), reinterpret_cast<const C *>(e.Eh),
          eval_src, u, e.k, n1, nh, ss);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      continue;
    }
    if (D == 3 && lr.tensor == 2 && sizeof(R) == 4) {  // stages 2-3 on the tensor cores
      const bool small_n = 2 * ((n1 + 7) / 8) <= 8;
      auto tk = lr.rows <= 4 ? (small_n ? eval4_kernel<8, 4> : eval4_kernel<kNbtMax, 4>)
                : lr.rows <= 8 ? (small_n ? eval4_kernel<8, 8> : eval4_kernel<kNbtMax, 8>)
                               : (small_n ? eval4_kernel<8, 16> : eval4_kernel<kNbtMax, 16>);
      const int rows4 = lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16;
      if ((err = cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lr.smem)) != cudaSuccess)
        return err;
      tk<<<dim3((unsigned)lr.count, (unsigned)((lr.K + rows4 - 1) / rows4)), 256, lr.smem, es.next()>>>(
          e.e2_blocks + lr.first, e.eval_leaves, reinterpret_cast<const float2 *>(e.Ef),
          reinterpret_cast<const float2 *>(e.Eh), reinterpret_cast<const float2 *>(eval_src), u, e.k, n1, nh, ss);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      continue;
    }
    // lr.rows rows of a block per CTA (tcgen05 ranges without the operand copy or the padded layout
    // of the expansions, as in the allocation-free call, take the CUDA-core kernel)
    const bool tc_fallback = lr.tensor == 4 || lr.tensor == 7;
    auto kern = (lr.tensor && !tc_fallback) ? (lr.rows <= 4   ? eval2_kernel<D, R, 4, true>
                             : lr.rows <= 8 ? eval2_kernel<D, R, 8, true>
                                            : eval2_kernel<D, R, 16, true>)
                          : (lr.rows <= 4   ? eval2_kernel<D, R, 4>
                             : lr.rows <= 8 ? eval2_kernel<D, R, 8>
                                            : eval2_kernel<D, R, 16>);
    const int rows = lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16;
    const unsigned chunks = (unsigned)((lr.K + rows - 1) / rows);
    const size_t esm2 = tc_fallback ? eval2_bytes(D, lr.K, n1, nh, sizeof(C), rows) : lr.smem;
    if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm2)) != cudaSuccess)
      return err;
    kern<<<dim3((unsigned)lr.count, chunks), 256, esm2, es.next()>>>(
        e.e2_blocks + lr.first, e.eval_leaves, reinterpret_cast<const C *>(e.Ef), reinterpret_cast<const C *>(e.Eh),
        eval_src, u, e.k, n1, nh, ss);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if ((err = es.join()) != cudaSuccess) return err;
  mark(4, 1);
  if (e.n_near_pairs > 0 && !near_aside) {
    if ((err = launch_near(st)) != cudaSuccess) return err;
  }
  if (near_aside && (err = cudaStreamWaitEvent(st, e.join_ev[0], 0)) != cudaSuccess) return err;
  return cudaSuccess;
}

int launches_per_transform(const ExecDesc &e) {
  int n = 0;
  n += (e.d == 3 && e.prec == 1 && e.n_pack > 0);  // sigma packing
  n += (e.d == 3 && e.prec == 1 && e.n_psi_tc_slots > 0);  // tcgen05 operand copy of the expansions
  if (e.d == 3 && e.prec == 0 && e.oz) {  // sliced FP64 tensor-core stages
    for (int kind = 0; kind < 6; ++kind) n += 2 * (e.oz_njobs[kind] > 0);  // slicing + products
  } else {
    n += (e.n_f1 > 0) + (int)e.f2_ranges.size() + (e.n_e1 > 0) + (int)e.e2_ranges.size();  // form + evaluate
  }
  for (const ShiftStep &s : e.merge) n += s.n > 0;
  for (const ShiftStep &s : e.push) n += s.n > 0;
  if (!e.fourier && e.n_gather > 0) n += 1;
  if (e.n_near_pairs > 0) n += 1;
  return n;
}

// ----------------------------------------------------------------------------- persistent batched execution
//
// Many independent transforms in ONE launch: every CTA of a persistent grid pops items from a device
// work queue, one item being one CTA's share of a kernel launch of one transform (a (transform,
// phase, block, row chunk) unit), runs it with the same device code as that kernel (the *_body
// functions), and counts it done in its transform's counter for the phase.  Items of a phase wait,
// with a bounded spin, until their transform's previous phase is complete (the queue lists every
// phase of every transform before the next phase, so an item only ever waits for items popped
// before it, by CTAs that are running).  A wait that runs out records kBatchTimeout in the batch's
// status word and the item is skipped (its result is then wrong, and the status says so), so
// nothing can hang.  Phases: 0 clear u / phi, 1 pack the FP32 density, 2 form, 3 gather,
// 4 evaluation, 5 near field (needs phase 0 only).  The items use the CUDA-core kernels (the tcgen05
// ranges of a plan take their CUDA-core fallbacks), the plain expansion layout and, for FP64 plans,
// the per-anchor gather (the run form's registers would lower the persistent kernel's occupancy).
struct BatchDesc {
  int d, k, n1, nh, f32, Kmax_f1;
  int64_t ss, n_points, phi_elems;
  const double *sigma;
  double *u;
  void *phi, *psi, *eval_src;
  float *sigp;
  const Block *blocks, *f1_blocks, *f2_blocks, *e1_blocks, *e2_blocks;
  const int32_t *f2_gptr, *pack_block;
  const int64_t *block_leaves, *eval_leaves;
  const void *Ff, *Fh, *Ef, *Eh, *Pf, *Ph;
  const int32_t *gather_dst;
  const int64_t *gather_ptr;
  const GatherSrc *gather_src;
  const GatherSeg *gather_segs;
  const NearPair *near_pairs;
  const double *near_tab;
  const int16_t *near_band;
};

struct BatchItem {
  int16_t kind, var;  // body and template variant
  int16_t phase, dep; // the phase counter it completes, the one it waits for (-1: none)
  int32_t t;          // transform
  int32_t first;      // first group / block of the item's launch range
  int32_t bx, by;     // its block index in that launch
  int32_t need;       // items the dep counter must count
  int32_t nb;         // consecutive block indices bx .. bx + nb - 1 of the launch
};

constexpr int kBatchPhases = 6;
constexpr int kZeroChunk = 1 << 15;     // elements cleared per item
constexpr int kBatchTimeout = 1;        // status word value of a wait that ran out
enum : int16_t { BK_ZERO_U = 1, BK_ZERO_PHI, BK_PACK, BK_FORM1, BK_FORM2, BK_FORM3, BK_FORM4, BK_GATHER, BK_GATHER2,
                 BK_EVAL1, BK_EVAL2, BK_EVAL5, BK_EVAL4, BK_NEAR, BK_NEVER };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int D, typename R>
__device__ __forceinline__ void batch_item_typed(const BatchDesc &b, const BatchItem &w) {
  using C = typename C2T<R>::T;
  const C *Ff = static_cast<const C *>(b.Ff), *Fh = static_cast<const C *>(b.Fh);
  const C *Ef = static_cast<const C *>(b.Ef), *Eh = static_cast<const C *>(b.Eh);
  const C *Pf = static_cast<const C *>(b.Pf), *Ph = static_cast<const C *>(b.Ph);
  C *phi = static_cast<C *>(b.phi), *psi = static_cast<C *>(b.psi);
  const C *src = static_cast<const C *>(b.eval_src);
  const int v = w.var >> 2;
  switch (w.kind) {
    case BK_FORM1:
      form_body<D, R>(b.f1_blocks, b.block_leaves, b.sigma, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss, b.Kmax_f1, w.bx, w.by);
      break;
    case BK_FORM2:
      if constexpr (D == 2)
        form2_body<2, R>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss,
                         w.bx, w.by);
      break;
    case BK_FORM3:
      if constexpr (D == 3)
        form3_body<R, false>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, Ff, Fh, phi, b.k, b.n1, b.nh,
                             b.ss, w.bx, w.by);
      break;
    case BK_FORM4:
      if constexpr (D == 3 && sizeof(R) == 4) {
        const float *sp = (v & 4) ? nullptr : b.sigp;
        if (v & 1) {
          if (v & 2) form4_body<8, true>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, sp, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss, w.bx, 0);
          else form4_body<8, false>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, sp, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss, w.bx, 0);
        } else {
          if (v & 2) form4_body<kNbtMax, true>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, sp, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss, w.bx, 0);
          else form4_body<kNbtMax, false>(b.f2_blocks, b.f2_gptr + w.first, b.block_leaves, b.sigma, sp, Ff, Fh, phi, b.k, b.n1, b.nh, b.ss, w.bx, 0);
        }
      }
      break;
    case BK_GATHER:
      gather_body<D, R>(b.gather_dst, b.gather_ptr, b.gather_src, Pf, Ph, phi, psi, b.n1, b.nh, b.ss, 0, w.bx, w.by);
      break;
    case BK_GATHER2:
      if constexpr (sizeof(R) == 4)
        gather2_body<D, R, kSegW>(b.gather_segs, Pf, Ph, phi, psi, b.n1, b.nh, b.ss, 0, w.bx, w.by);
      break;
    case BK_EVAL1:
      eval_body<D, R>(b.e1_blocks, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
      break;
    case BK_EVAL2: {
      const Block *bl = b.e2_blocks + w.first;
      if (v == 0) eval2_body<D, R, 4, false>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
      else if (v == 1) eval2_body<D, R, 8, false>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
      else eval2_body<D, R, 16, false>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
      break;
    }
    case BK_EVAL5:
      if constexpr (D == 3 && sizeof(R) == 8) {
        const Block *bl = b.e2_blocks + w.first;
        switch (v) {
          case 0: eval5_body<R, 1>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by); break;
          case 1: eval5_body<R, 2>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by); break;
          case 2: eval5_body<R, 4>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by); break;
          case 3: eval5_body<R, 8>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by); break;
          default: eval5_body<R, 16>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by); break;
        }
      }
      break;
    case BK_EVAL4:
      if constexpr (D == 3 && sizeof(R) == 4) {
        const Block *bl = b.e2_blocks + w.first;
        const int km = v >> 1;
        if (v & 1) {
          if (km == 0) eval4_body<8, 4>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
          else if (km == 1) eval4_body<8, 8>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
          else eval4_body<8, 16>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
        } else {
          if (km == 0) eval4_body<kNbtMax, 4>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
          else if (km == 1) eval4_body<kNbtMax, 8>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
          else eval4_body<kNbtMax, 16>(bl, b.eval_leaves, Ef, Eh, src, b.u, b.k, b.n1, b.nh, b.ss, w.bx, w.by);
        }
      }
      break;
    case BK_NEAR:
      near2_body<D>(b.near_pairs, b.near_tab, b.near_band, b.sigma, b.u, b.k, w.bx, 0);
      break;
    default:
      break;
  }
}

__global__ void __launch_bounds__(256, 2) batch_persistent_kernel(const BatchItem *__restrict__ items, int n_items,
                                                                  const BatchDesc *__restrict__ descs,
                                                                  unsigned *__restrict__ counters,
                                                                  unsigned *__restrict__ head, int *__restrict__ status,
                                                                  long long wait_clocks) {
  __shared__ int s_item, s_skip;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem w = items[it];
    if (tid == 0) {
      int skip = 0;
      if (w.dep >= 0) {
        const unsigned *c = counters + (size_t)w.t * kBatchPhases + w.dep;
        const long long t0 = clock64();
        while (ld_acquire_u32(c) < (unsigned)w.need) {
          if (clock64() - t0 > wait_clocks) {  // the phase it needs never completed: report, skip
            atomicMax(status, kBatchTimeout);
            skip = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      s_skip = skip;
    }
    __syncthreads();
    const BatchItem w0 = w;
    for (int j = 0; j < w0.nb && !s_skip; ++j) {
      if (j > 0) __syncthreads();  // the previous block's shared memory is free
      BatchItem w = w0;
      w.bx = w0.bx + j;
      const BatchDesc &b = descs[w.t];
      if (w.kind == BK_ZERO_U || w.kind == BK_ZERO_PHI) {
        // clear a chunk of u (doubles) or of the outgoing expansions (complex values, as uint2 words
        // of 8 bytes: FP32 complex, or halves of an FP64 complex)
        const int64_t n = w.kind == BK_ZERO_U ? b.n_points : b.phi_elems * (b.f32 ? 1 : 2);
        const int64_t lo = (int64_t)w.bx * kZeroChunk, hi = min(n, lo + kZeroChunk);
        uint2 *p = w.kind == BK_ZERO_U ? reinterpret_cast<uint2 *>(b.u) : static_cast<uint2 *>(b.phi);
        for (int64_t e = lo + tid; e < hi; e += blockDim.x) p[e] = make_uint2(0u, 0u);
      } else if (w.kind == BK_PACK) {
        sigma_pack_body(b.blocks, b.pack_block, b.block_leaves, b.sigma, b.sigp, b.k, w.bx, 0);
      } else {
        const bool f32 = (w.var & 1) != 0, d3 = (w.var & 2) != 0;
        if (d3) {
          if (f32) batch_item_typed<3, float>(b, w);
          else batch_item_typed<3, double>(b, w);
        } else {
          if (f32) batch_item_typed<2, float>(b, w);
          else batch_item_typed<2, double>(b, w);
        }
      }
    }
    __syncthreads();  // the item's writes are done (and s_item may be rewritten)
    if (tid == 0) {
      __threadfence();
      atomicAdd(counters + (size_t)w.t * kBatchPhases + w.phase, 1u);
    }
  }
}

struct BatchQueue {
  std::vector<BatchItem> items;
  std::vector<BatchDesc> descs;
  size_t smem = 0;
  BatchItem *d_items = nullptr;
  BatchDesc *d_descs = nullptr;
  unsigned *d_counters = nullptr;  // [n][kBatchPhases], then the queue head
  int *d_status = nullptr;
  int grid = 0;
  std::vector<const double *> sig;
  std::vector<double *> u;
  ~BatchQueue() {
    cudaFree(d_items);
    cudaFree(d_descs);
    cudaFree(d_counters);
    cudaFree(d_status);
  }
};

namespace {
// The launches of one transform (fused mode) as queue items, following run_typed's choices with the
// CUDA-core kernel wherever it takes a tcgen05 one.  Returns nullptr or why the plan cannot be queued.
const char *queue_transform(const ExecDesc &e, int t, std::vector<BatchItem> (&ph)[kBatchPhases], size_t &smem,
                            BatchDesc &bd) {
  if (!e.merge.empty() || !e.push.empty()) return "hierarchical mode";
  if (e.tc64) return "FP64 tensor-core precision";
  const int D = e.d, n1 = e.n1, nh = e.nh;
  const bool f32 = e.prec == 1;
  const int vbase = (f32 ? 1 : 0) | (D == 3 ? 2 : 0);
  const size_t csz = f32 ? sizeof(float2) : sizeof(double2);
  int count[kBatchPhases] = {};
  auto add = [&](int phase, int16_t kind, int var, int first, int gx, int gy, size_t sm) {
    // a few consecutive blocks of the launch per item (fewer queue pops and dependency checks)
    const int g = gx >= 16 ? 4 : gx >= 8 ? 2 : 1;
    for (int y = 0; y < gy; ++y)
      for (int x = 0; x < gx; x += g) {
        BatchItem w{};
        w.kind = kind;
        w.var = (int16_t)(vbase | (var << 2));
        w.phase = (int16_t)phase;
        w.t = t;
        w.first = first;
        w.bx = x;
        w.by = y;
        w.nb = std::min(g, gx - x);
        ph[phase].push_back(w);
        ++count[phase];
      }
    smem = std::max(smem, sm);
  };
  const int64_t ss = e.slot_size;
  if (e.zero_u) add(0, BK_ZERO_U, 0, 0, (int)((e.n_points + kZeroChunk - 1) / kZeroChunk), 1, 0);
  const int64_t phi_words = e.n_phi_slots * ss * (f32 ? 1 : 2);
  if (e.n_blocks > 0) add(0, BK_ZERO_PHI, 0, 0, (int)((phi_words + kZeroChunk - 1) / kZeroChunk), 1, 0);
  if (D == 3 && f32 && e.sigp != nullptr && e.n_pack > 0) add(1, BK_PACK, 0, 0, (int)e.n_pack, 1, 0);
  if (e.n_f1 > 0) add(2, BK_FORM1, 0, 0, (int)e.n_f1, nh, form_smem_bytes(D, e.Kmax_f1, n1, f32));
  for (const LaunchRange &lr : e.f2_ranges) {
    const int chunks = (nh + kSc - 1) / kSc;
    if (D == 3 && f32 && (lr.tensor == 7 || lr.tensor == 1)) {
      const bool big = lr.K > 16, small_n = n1_pad8(n1) / 4 <= 8;
      // tcgen05 ranges: the register-tiled form, reading sigma itself (their blocks' packed copy
      // is in the tcgen05 order)
      const bool own = lr.tensor == 7 || e.sigp == nullptr;
      const size_t sm = lr.tensor == 7 ? (big ? form4b_bytes(lr.K, n1) : form4_bytes(1, lr.K, n1)) : lr.smem;
      add(2, BK_FORM4, (small_n ? 1 : 0) | ((lr.tensor == 7 ? big : lr.big) ? 2 : 0) | (own ? 4 : 0), lr.first,
          lr.count * chunks, 1, sm);
    } else if (D == 3) {
      add(2, BK_FORM3, 0, lr.first, lr.count, chunks, lr.smem);
    } else {
      add(2, BK_FORM2, 0, lr.first, lr.count, nh, lr.smem);
    }
  }
  if (!e.fourier && e.n_gather > 0) {
    if (e.n_gather_segs > 0 && f32) {
      add(3, BK_GATHER2, 0, 0, (int)e.n_gather_segs, (int)((ss + 255) / 256), 0);
    } else {
      add(3, BK_GATHER, 0, 0, (int)e.n_gather, (int)((ss + 256 * kGatherMpt - 1) / (256 * kGatherMpt)), 0);
    }
  }
  if (e.n_e1 > 0) add(4, BK_EVAL1, 0, 0, (int)e.n_e1, e.Kmax_e1, eval_smem_bytes(D, e.Kmax_e1, n1, f32));
  for (const LaunchRange &lr : e.e2_ranges) {
    if (lr.tensor == 1) return "tensor-core evaluation variant";
    const int rows = lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16, kmv = rows == 4 ? 0 : rows == 8 ? 1 : 2;
    if (lr.tensor == 3) {
      if (f32) return "FP32 half-range-last evaluation";
      const int rc = lr.rows <= 1 ? 1 : lr.rows <= 2 ? 2 : lr.rows <= 4 ? 4 : lr.rows <= 8 ? 8 : 16;
      const int rv = rc == 1 ? 0 : rc == 2 ? 1 : rc == 4 ? 2 : rc == 8 ? 3 : 4;
      add(4, BK_EVAL5, rv, lr.first, lr.count, (lr.K + rc - 1) / rc, lr.smem);
    } else if (lr.tensor == 2) {
      const bool small_n = 2 * ((n1 + 7) / 8) <= 8;
      add(4, BK_EVAL4, (small_n ? 1 : 0) | (kmv << 1), lr.first, lr.count, (lr.K + rows - 1) / rows, lr.smem);
    } else {
      // the CUDA-core whole-block kernel, also for the tcgen05 ranges (4, 7)
      const size_t sm = (lr.tensor == 4 || lr.tensor == 7) ? eval2_bytes(D, lr.K, n1, nh, csz, rows) : lr.smem;
      add(4, BK_EVAL2, kmv, lr.first, lr.count, (lr.K + rows - 1) / rows, sm);
    }
  }
  if (e.n_near_pairs > 0) {
    const int np = D == 3 ? e.k * e.k * e.k : e.k * e.k;
    const size_t nsm = sizeof(double) * (3 * (size_t)np + (size_t)D * e.k * e.k) + sizeof(int16_t) * 2 * D * e.k;
    add(5, BK_NEAR, 0, 0, (int)e.n_near_pairs, 1, nsm);
  }
  // dependencies: each phase waits for the latest earlier phase of the chain 0 -> 1 -> 2 -> 3 -> 4 that
  // has items; the near field for phase 0 only
  auto dep_of = [&](int phase) -> int {
    if (phase == 5) return count[0] ? 0 : -1;
    for (int q = phase - 1; q >= 0; --q)
      if (count[q]) return q;
    return -1;
  };
  for (int q = 0; q < kBatchPhases; ++q) {
    const int dq = dep_of(q);
    for (size_t i = ph[q].size() - count[q]; i < ph[q].size(); ++i) {
      ph[q][i].dep = (int16_t)dq;
      ph[q][i].need = dq >= 0 ? count[dq] : 0;
    }
  }
  bd = BatchDesc{};
  bd.d = D; bd.k = e.k; bd.n1 = n1; bd.nh = nh; bd.f32 = f32; bd.Kmax_f1 = e.Kmax_f1;
  bd.ss = ss; bd.n_points = e.n_points; bd.phi_elems = e.n_phi_slots * ss;
  bd.phi = e.phi; bd.psi = e.psi; bd.eval_src = (!e.fourier && e.n_gather > 0) ? e.psi : e.phi;
  bd.sigp = e.sigp;
  bd.blocks = e.blocks; bd.f1_blocks = e.f1_blocks; bd.f2_blocks = e.f2_blocks; bd.e1_blocks = e.e1_blocks;
  bd.e2_blocks = e.e2_blocks; bd.f2_gptr = e.f2_gptr; bd.pack_block = e.pack_block;
  bd.block_leaves = e.block_leaves; bd.eval_leaves = e.eval_leaves;
  bd.Ff = e.Ff; bd.Fh = e.Fh; bd.Ef = e.Ef; bd.Eh = e.Eh; bd.Pf = e.Pf; bd.Ph = e.Ph;
  bd.gather_dst = e.gather_dst; bd.gather_ptr = e.gather_ptr; bd.gather_src = e.gather_src;
  bd.gather_segs = e.gather_segs;
  bd.near_pairs = e.near_pairs; bd.near_tab = e.near_tab; bd.near_band = e.near_band;
  return nullptr;
}
}  // namespace

cudaError_t batch_queue_create(const std::vector<const ExecDesc *> &plans, BatchQueue **out, const char **why) {
  *out = nullptr;
  *why = nullptr;
  auto *q = new (std::nothrow) BatchQueue();
  if (!q) return cudaErrorMemoryAllocation;
  std::vector<BatchItem> ph[kBatchPhases];
  q->descs.resize(plans.size());
  for (size_t t = 0; t < plans.size(); ++t) {
    const char *w = queue_transform(*plans[t], (int)t, ph, q->smem, q->descs[t]);
    if (w) {
      *why = w;
      delete q;
      return cudaSuccess;
    }
  }
  // phase-major order: every transform's clears, packs, forms, near fields, gathers, evaluations
  for (int p : {0, 1, 2, 5, 3, 4}) q->items.insert(q->items.end(), ph[p].begin(), ph[p].end());
  if (q->items.size() > (size_t)INT32_MAX) { delete q; return cudaErrorInvalidValue; }
  cudaError_t err = cudaFuncSetAttribute(batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)q->smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, 256, q->smem);
  if (err == cudaSuccess) err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess && per_sm < 1) err = cudaErrorInvalidConfiguration;
  q->grid = (int)std::min<size_t>(q->items.size(), (size_t)std::max(1, per_sm) * (size_t)sms);
  if (err == cudaSuccess) err = cudaMalloc(&q->d_items, sizeof(BatchItem) * std::max<size_t>(1, q->items.size()));
  if (err == cudaSuccess) err = cudaMalloc(&q->d_descs, sizeof(BatchDesc) * std::max<size_t>(1, q->descs.size()));
  if (err == cudaSuccess) err = cudaMalloc(&q->d_counters, sizeof(unsigned) * (plans.size() * kBatchPhases + 1));
  if (err == cudaSuccess) err = cudaMalloc(&q->d_status, sizeof(int));
  if (err == cudaSuccess && !q->items.empty())
    err = cudaMemcpy(q->d_items, q->items.data(), sizeof(BatchItem) * q->items.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemset(q->d_status, 0, sizeof(int));
  if (err != cudaSuccess) { delete q; return err; }
  q->sig.assign(plans.size(), nullptr);
  q->u.assign(plans.size(), nullptr);
  *out = q;
  return cudaSuccess;
}

cudaError_t batch_queue_run(BatchQueue *q, const double *const *sigma, double *const *u, cudaStream_t st,
                            long long wait_clocks) {
  bool same = true;
  for (size_t t = 0; t < q->descs.size(); ++t) {
    if (q->sig[t] != sigma[t] || q->u[t] != u[t]) same = false;
    q->sig[t] = sigma[t];
    q->u[t] = u[t];
    q->descs[t].sigma = sigma[t];
    q->descs[t].u = u[t];
  }
  cudaError_t err = cudaSuccess;
  if (!same)  // the descriptors hold the buffers: uploaded when a pointer changes
    err = cudaMemcpyAsync(q->d_descs, q->descs.data(), sizeof(BatchDesc) * q->descs.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess)
    err = cudaMemsetAsync(q->d_counters, 0, sizeof(unsigned) * (q->descs.size() * kBatchPhases + 1), st);
  if (err != cudaSuccess) return err;
  if (q->items.empty()) return cudaSuccess;
  batch_persistent_kernel<<<q->grid, 256, q->smem, st>>>(q->d_items, (int)q->items.size(), q->d_descs, q->d_counters,
                                                         q->d_counters + q->descs.size() * kBatchPhases, q->d_status,
                                                         wait_clocks);
  return cudaGetLastError();
}

cudaError_t batch_queue_status(BatchQueue *q, int *status) {
  int v = 0;
  cudaError_t err = cudaMemcpy(&v, q->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && v != 0) err = cudaMemset(q->d_status, 0, sizeof(int));
  *status = v;
  return err;
}

size_t batch_queue_items(const BatchQueue *q) { return q->items.size(); }
int batch_queue_grid(const BatchQueue *q) { return q->grid; }
void batch_queue_destroy(BatchQueue *q) { delete q; }

// A queue of one item whose dependency (a counter nothing increments) cannot be met: its bounded wait
// (wait_clocks) runs out and the status word reports it.  Faults nothing, hangs nothing.
cudaError_t selftest_batch_timeout(int *status) {
  BatchItem w{};
  w.kind = BK_NEVER;
  w.phase = 1;
  w.dep = 0;
  w.need = 1;
  w.nb = 1;
  BatchItem *di = nullptr;
  BatchDesc *dd = nullptr;
  unsigned *dc = nullptr;
  int *ds = nullptr;
  cudaError_t err = cudaMalloc(&di, sizeof(BatchItem));
  if (err == cudaSuccess) err = cudaMalloc(&dd, sizeof(BatchDesc));
  if (err == cudaSuccess) err = cudaMalloc(&dc, sizeof(unsigned) * (kBatchPhases + 1));
  if (err == cudaSuccess) err = cudaMalloc(&ds, sizeof(int));
  if (err == cudaSuccess) err = cudaMemcpy(di, &w, sizeof(BatchItem), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemset(dd, 0, sizeof(BatchDesc));
  if (err == cudaSuccess) err = cudaMemset(dc, 0, sizeof(unsigned) * (kBatchPhases + 1));
  if (err == cudaSuccess) err = cudaMemset(ds, 0, sizeof(int));
  if (err == cudaSuccess) {
    batch_persistent_kernel<<<1, 256, 0>>>(di, 1, dd, dc, dc + kBatchPhases, ds, 1LL << 21);  // about a millisecond
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(status, ds, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(di);
  cudaFree(dd);
  cudaFree(dc);
  cudaFree(ds);
  return err;
}

cudaError_t run_transform(const ExecDesc &e, const double *sigma, double *u, cudaStream_t stream) {
  if (e.d == 3) return e.prec ? run_typed<3, float>(e, sigma, u, stream) : run_typed<3, double>(e, sigma, u, stream);
  return e.prec ? run_typed<2, float>(e, sigma, u, stream) : run_typed<2, double>(e, sigma, u, stream);
}

cudaError_t set_check_ranges(const void *const *base, const size_t *bytes, int n, cudaStream_t st) {
#ifdef FGT_CHECKED
  CheckRanges r{};
  r.n = n < kCheckRanges ? n : kCheckRanges;
  for (int i = 0; i < r.n; ++i) {
    r.lo[i] = static_cast<const char *>(base[i]);
    r.hi[i] = r.lo[i] + bytes[i];
  }
  return cudaMemcpyToSymbolAsync(g_check_ranges, &r, sizeof(r), 0, cudaMemcpyHostToDevice, st);
#else
  (void)base, (void)bytes, (void)n, (void)st;
  return cudaSuccess;
#endif
}

cudaError_t read_check(unsigned *site, unsigned *count, int *checked) {
#ifdef FGT_CHECKED
  *checked = 1;
  cudaError_t err = cudaMemcpyFromSymbol(site, g_check_word, sizeof(unsigned));
  if (err == cudaSuccess) err = cudaMemcpyFromSymbol(count, g_check_count, sizeof(unsigned));
  const unsigned zero = 0;
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(unsigned));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_check_count, &zero, sizeof(unsigned));
  return err;
#else
  *checked = 0;
  *site = *count = 0;
  return cudaSuccess;
#endif
}

cudaError_t selftest_tc_timeout() {
  wait_timeout_selftest_kernel<<<1, 1>>>(1LL << 21);  // about a millisecond
  cudaError_t err = cudaGetLastError();
  return err != cudaSuccess ? err : cudaDeviceSynchronize();
}

cudaError_t read_tc_status(int *status) {
  int v = 0, v7 = 0, vf = 0;
  cudaError_t err = cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemcpyFromSymbol(&v7, g_tc7_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemcpyFromSymbol(&vf, g_tcf_status, sizeof(int));
  if (err != cudaSuccess) return err;
  const int zero = 0;
  if (v != 0 && (err = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int))) != cudaSuccess) return err;
  if (v7 != 0 && (err = cudaMemcpyToSymbol(g_tc7_status, &zero, sizeof(int))) != cudaSuccess) return err;
  if (vf != 0 && (err = cudaMemcpyToSymbol(g_tcf_status, &zero, sizeof(int))) != cudaSuccess) return err;
  int vo = 0;
  if ((err = read_oz_status(&vo)) != cudaSuccess) return err;
  *status = std::max(std::max(v, vo), std::max(v7, vf));
  return cudaSuccess;
}

size_t form7_smem_bytes(int K) { return f7::smem_bytes(K); }

cudaError_t encode_sig_maps(ExecDesc &e, int64_t total_floats, const bool *used) {
  // the packed density as rows of K floats (K = 8, 16, 32), one tensor map each, with the swizzle
  // of a K-float row so that a 128-row box lands in the tensor cores' K-major layout
  using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (err != cudaSuccess) return err;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  Encode encode = reinterpret_cast<Encode>(fn);
  const int Ks[3] = {8, 16, 32};
  const CUtensorMapSwizzle sw[3] = {CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_SWIZZLE_128B};
  for (int i = 0; i < 3; ++i) {
    if (!used[i]) continue;
    const cuuint64_t K = (cuuint64_t)Ks[i];
    const cuuint64_t dims[2] = {K, (cuuint64_t)(total_floats / Ks[i])};
    const cuuint64_t strides[1] = {K * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)K, 128}, estr[2] = {1, 1};
    const CUresult r = encode(&e.sig_map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, e.sigp, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, sw[i], CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

size_t eval7_smem_bytes(int K) { return e7::smem_bytes(K); }
int eval7_pitch() { return e7::kP; }

cudaError_t encode_psi_map(ExecDesc &e) {
  // the padded expansions as a 3D FP32 tensor: (64 floats of m1 re/im, nh * 32 rows (m3, m2), slots)
  using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (err != cudaSuccess) return err;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<Encode>(fn);
  }
  const cuuint64_t P = (cuuint64_t)e.psi_pitch;
  const cuuint64_t dims[3] = {2 * P, (cuuint64_t)e.nh * P, (cuuint64_t)e.n_psi_slots};
  const cuuint64_t strides[2] = {2 * P * sizeof(float), (cuuint64_t)e.nh * P * 2 * P * sizeof(float)};
  const cuuint32_t box[3] = {32, 128, 1}, estr[3] = {1, 1, 1};
  const CUresult r = encode(&e.psi_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, e.psi, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
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
  const size_t psi_off = (phi_bytes + 255) & ~(size_t)255;
  if (psi_off + psi_bytes > kNoallocScratchBytes) return cudaErrorInvalidValue;
  ExecDesc f = e;
  f.phi = base;
  f.psi = static_cast<unsigned char *>(base) + psi_off;
  f.sigp = nullptr;  // no packed sigma: the form kernels read sigma itself
  f.sig_order = 0;
  f.phi_stored = 0;  // and the CUDA-core forms add into a cleared slot
  f.psi_tc = nullptr;  // no operand copy of the expansions: the CUDA-core evaluation throughout
  f.n_psi_tc_slots = 0;
  f.psi_pitch = 0;     // and the plain expansion layout (no tensor map over the scratch array)
  f.psi_map_ready = 0;
  f.sig_maps_ready = 0;
  f.oz = 0;            // no sliced tensor-core stages (their intermediates live in the plan's workspace)
  f.oz_x = f.oz_y = nullptr;
  f.events = nullptr;
  return run_transform(f, sigma, u, stream);
}

// ----------------------------------------------------------------------------- tree refinement / coarsening
//
// Error monitor of Algorithms 3, 5 and 6 (eq. funerr): the tensor Legendre coefficients c of a
// box's interpolant (val -> pol, Definition val2poldef: T[n][j] = (2n+1)/2 w_j P_n(eta_j) per axis)
// and e = sqrt(mean of |c_alpha|^2 over ||alpha||_2 >= k).  Also returns the box's quadrature
// sum of v^2 (weights of the reference box [-1,1]^d) for the norm the criterion is relative to.

// Legendre values P_0..P_{k-1} at x by the three-term recurrence.
__device__ inline void legendre_all(int k, double x, double *P) {
  P[0] = 1.0;
  if (k > 1) P[1] = x;
  for (int n = 2; n < k; ++n) P[n] = ((2 * n - 1) * x * P[n - 1] - (n - 1) * P[n - 2]) / n;
}

__global__ void __launch_bounds__(256) leaf_error_kernel(int d, int k, GLRule gl, const double *__restrict__ vals,
                                                         double *__restrict__ err, double *__restrict__ sumsq) {
  extern __shared__ double sme[];
  const int kk = k * k, np = d == 3 ? kk * k : kk;
  double *V = sme, *A = V + np, *B = A + np, *T = B + np;  // T: [k][k]
  const double *v = vals + (int64_t)blockIdx.x * np;
  for (int e = threadIdx.x; e < np; e += blockDim.x) V[e] = v[e];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double P[kMaxLeafK];
    legendre_all(k, gl.x[j], P);
    for (int n = 0; n < k; ++n) T[n * k + j] = 0.5 * (2 * n + 1) * gl.w[j] * P[n];
  }
  __syncthreads();
  // c = (T x T (x T)) v, axis 1 first (node index j_1 fastest)
  double *src = V, *dst = A;
  for (int a = 0; a < d; ++a) {
    const int stride = a == 0 ? 1 : (a == 1 ? k : kk);
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      const int na = (e / stride) % k, base = e - na * stride;
      double acc = 0.0;
      for (int j = 0; j < k; ++j) acc = fma(T[na * k + j], src[base + j * stride], acc);
      dst[e] = acc;
    }
    __syncthreads();
    src = dst;
    dst = (dst == A) ? B : A;
  }
  // tail and quadrature sums
  __shared__ double red[2][256];
  __shared__ int cnt[256];
  double tail = 0.0, sq = 0.0;
  int ntail = 0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    const int a1 = e % k, a2 = (e / k) % k, a3 = d == 3 ? e / kk : 0;
    if (a1 * a1 + a2 * a2 + a3 * a3 >= k * k) {
      tail += src[e] * src[e];
      ++ntail;
    }
    double w = gl.w[a1] * gl.w[a2] * (d == 3 ? gl.w[a3] : 1.0);
    sq += w * V[e] * V[e];
  }
  red[0][threadIdx.x] = tail;
  red[1][threadIdx.x] = sq;
  cnt[threadIdx.x] = ntail;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      red[0][threadIdx.x] += red[0][threadIdx.x + off];
      red[1][threadIdx.x] += red[1][threadIdx.x + off];
      cnt[threadIdx.x] += cnt[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    err[blockIdx.x] = cnt[0] > 0 ? sqrt(red[0][0] / cnt[0]) : 0.0;
    if (sumsq) sumsq[blockIdx.x] = red[1][0];
  }
}

// Algorithm 6: the values of a parent box at its k^d nodes from the interpolants of its 2^d
// children (child c holds the half (c >> a) & 1 along axis a): a parent node in child c's half
// is the child's Lagrange interpolant at the node's child-local coordinate 2 eta -/+ 1, applied
// axis by axis.  One CTA per parent.
__global__ void __launch_bounds__(256) merge_children_kernel(int d, int k, GLRule gl,
                                                             const int64_t *__restrict__ child_rows,
                                                             const double *__restrict__ vals,
                                                             double *__restrict__ parent) {
  extern __shared__ double smm[];
  const int kk = k * k, np = d == 3 ? kk * k : kk, nc = 1 << d;
  double *M = smm;                 // [2][k][k]: M[h][t][j] = l_j(2 eta_t - 1 + 2 (1 - h) ... )
  double *A = M + 2 * kk, *B = A + np, *Cv = B + np;
  for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
    const int h = e / kk, t = (e / k) % k, j = e % k;
    const double s = h ? 2.0 * gl.x[t] - 1.0 : 2.0 * gl.x[t] + 1.0;  // child-local coordinate
    double l = 1.0;
    for (int m = 0; m < k; ++m)
      if (m != j) l *= (s - gl.x[m]) / (gl.x[j] - gl.x[m]);
    M[e] = l;
  }
  __syncthreads();
  double *out = parent + (int64_t)blockIdx.x * np;
  for (int c = 0; c < nc; ++c) {
    const double *v = vals + child_rows[(int64_t)blockIdx.x * nc + c] * np;
    for (int e = threadIdx.x; e < np; e += blockDim.x) Cv[e] = v[e];
    __syncthreads();
    double *src = Cv, *dst = A;
    for (int a = 0; a < d; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? k : kk), h = (c >> a) & 1;
      for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int ta = (e / stride) % k, base = e - ta * stride;
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(M[(h * k + ta) * k + j], src[base + j * stride], acc);
        dst[e] = acc;
      }
      __syncthreads();
      src = dst;
      dst = (dst == A) ? B : A;
    }
    // keep the parent nodes that lie in child c's half on every axis (the middle node of an odd
    // k goes to the upper half)
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      bool mine = true;
      for (int a = 0, r = e; a < d; ++a, r /= k) mine = mine && ((gl.x[r % k] >= 0.0) == (((c >> a) & 1) == 1));
      if (mine) out[e] = src[e];
    }
    __syncthreads();
  }
}

// Algorithm 3's density evaluation for a sum of Gaussians sigma(x) = sum_i a_i exp(-|x - c_i|^2 /
// alpha_i) (periodic: the minimum-image distance to each centre) at the k^d tensor Gauss-Legendre
// nodes of n boxes (level, integer coordinates); one CTA per box, node index j_1 fastest.
__global__ void __launch_bounds__(256) gauss_nodes_kernel(int d, int k, GLRule gl, const int32_t *__restrict__ level,
                                                          const int32_t *__restrict__ coord, int ng,
                                                          const double *__restrict__ gparams, int periodic,
                                                          double *__restrict__ vals) {
  const int np = d == 3 ? k * k * k : k * k;
  const int64_t b = blockIdx.x;
  const double L = ldexp(1.0, -level[b]);
  double c[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < d; ++a) c[a] = -0.5 + (coord[b * d + a] + 0.5) * L;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0, r = e; a < d; ++a, r /= k) x[a] = c[a] + 0.5 * L * gl.x[r % k];
    double v = 0.0;
    for (int i = 0; i < ng; ++i) {
      const double *g = gparams + (size_t)i * (d + 2);  // centre[d], alpha, amplitude
      double r2 = 0.0;
      for (int a = 0; a < d; ++a) {
        double dx = x[a] - g[a];
        if (periodic) dx -= rint(dx);
        r2 += dx * dx;
      }
      v += g[d + 1] * exp(-r2 / g[d]);
    }
    vals[b * np + e] = v;
  }
}

cudaError_t gauss_nodes(int d, int k, int64_t n, const int32_t *level, const int32_t *coord, int ng,
                        const double *gparams, int periodic, double *vals, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  GLRule gl;
  gl_rule(k, gl.x, gl.w);
  gauss_nodes_kernel<<<(unsigned)n, 256, 0, st>>>(d, k, gl, level, coord, ng, gparams, periodic, vals);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- point FGT (Algorithm 2)
//
// The discrete transform with tensor-product "proxy" grids in the cutoff-level boxes (Section 8's
// closing remark): the sources of a dense box are replaced by the values Q on a k_p^d Gauss-
// Legendre grid that reproduce every plane wave of the expansion (Q = the transpose of Lagrange
// interpolation at the sources), the box-FGT form / gather / evaluation kernels run on those grids,
// and the incoming expansion is interpolated from the grid to the targets.

// l_t(s), t < kp, by the barycentric formula: the k_p reciprocals 1/(s - x_t) come from one
// division and prefix / suffix products of the differences (batch inversion).  A point within
// 1e-100 of a node takes that node's unit vector (the formula's limit to double precision).
// Entries kp..KP-1 are zero.  l[t] is written at l[t * stride].
template <int KP>
__device__ inline void lagrange_row(const ProxyRule &pr, int kp, double s, double *l, int stride) {
  double p = 1.0;
  int hit = -1;
  for (int t = 0; t < kp; ++t) {
    const double dx = s - pr.x[t];
    if (fabs(dx) < 1e-100) hit = t;
    l[t * stride] = p;  // prod_{m < t} (s - x_m)
    p *= dx;
  }
  for (int t = kp; t < KP; ++t) l[t * stride] = 0.0;
  if (hit >= 0) {
    for (int t = 0; t < kp; ++t) l[t * stride] = (t == hit) ? 1.0 : 0.0;
    return;
  }
  double inv = 1.0 / p, den = 0.0;  // inv = 1 / prod_{m <= t} (s - x_m) going down
  for (int t = kp - 1; t >= 0; --t) {
    const double c = pr.bw[t] * (inv * l[t * stride]);
    inv *= s - pr.x[t];
    l[t * stride] = c;
    den += c;
  }
  const double sc = 1.0 / den;
  for (int t = 0; t < kp; ++t) l[t * stride] *= sc;
}

// The same into registers (fully unrolled over the padded order KP).
template <int KP>
__device__ inline void lagrange_reg(const ProxyRule &pr, int kp, double s, double (&l)[KP]) {
  double p = 1.0;
  int hit = -1;
#pragma unroll
  for (int t = 0; t < KP; ++t) {
    l[t] = 0.0;
    if (t < kp) {
      const double dx = s - pr.x[t];
      if (fabs(dx) < 1e-100) hit = t;
      l[t] = p;
      p *= dx;
    }
  }
  if (hit >= 0) {
#pragma unroll
    for (int t = 0; t < KP; ++t) l[t] = (t == hit) ? 1.0 : 0.0;
    return;
  }
  double inv = 1.0 / p, den = 0.0;
#pragma unroll
  for (int t = KP - 1; t >= 0; --t)
    if (t < kp) {
      const double c = pr.bw[t] * (inv * l[t]);
      inv *= s - pr.x[t];
      l[t] = c;
      den += c;
    }
  const double sc = 1.0 / den;
#pragma unroll
  for (int t = 0; t < KP; ++t) l[t] *= sc;
}

constexpr int kPointThreads = 128;
constexpr int kLChunk = 32;  // points whose Lagrange rows are staged in shared memory at once

// Anterpolation.  Grid: x = source segment (box seg[3s], sources [seg[3s+1], seg[3s+2])), y = block
// of kPointThreads rows of the box's grid.  In 3D a thread owns the row (t_3, t_2) and keeps its k_p
// values along t_1 in registers for the whole segment, so each source costs it one product
// a = q_j l_{t_3} l_{t_2} and k_p FMAs against the shared l_{t_1} row; in 2D (k_p rows) the block's
// threads form groups of k_p that take every G-th source.  The segment's sums are added into the
// box's (cleared) grid atomically, so a crowded box spreads over many CTAs.
template <int KP>
__global__ void __launch_bounds__(kPointThreads) point_anterp_kernel(int d, int kp, ProxyRule pr,
                                                                     const int64_t *__restrict__ seg,
                                                                     const double *__restrict__ s_local,
                                                                     const double *__restrict__ q_sorted,
                                                                     double *__restrict__ Q) {
  __shared__ double L[kLChunk][3][KP];
  __shared__ double qs[kLChunk];
  const int tid = threadIdx.x;
  int r, g, G;
  if (d == 3) {
    r = blockIdx.y * kPointThreads + tid;
    g = 0;
    G = 1;
  } else {
    G = kPointThreads / kp;
    g = tid / kp;
    r = tid - g * kp;
  }
  const bool active = d == 3 ? r < kp * kp : g < G;
  const int t2 = d == 3 ? r % kp : r, t3 = d == 3 ? r / kp : 0;
  const int64_t box = seg[3 * blockIdx.x], j0 = seg[3 * blockIdx.x + 1], j1 = seg[3 * blockIdx.x + 2];
  double acc[KP];
#pragma unroll
  for (int t = 0; t < KP; ++t) acc[t] = 0.0;
  for (int64_t c0 = j0; c0 < j1; c0 += kLChunk) {
    const int nc = (int)min((int64_t)kLChunk, j1 - c0);
    __syncthreads();
    for (int e = tid; e < nc * d; e += kPointThreads) {
      const int j = e / d, a = e - j * d;
      lagrange_row<KP>(pr, kp, s_local[(c0 + j) * d + a], &L[j][a][0], 1);
    }
    for (int j = tid; j < nc; j += kPointThreads) qs[j] = q_sorted[c0 + j];
    __syncthreads();
    if (!active) continue;
    for (int j = g; j < nc; j += G) {
      double a = qs[j] * L[j][1][t2];
      if (d == 3) a *= L[j][2][t3];
#pragma unroll
      for (int t = 0; t < KP; ++t) acc[t] = fma(a, L[j][0][t], acc[t]);
    }
  }
  if (!active) return;
  const int rows = d == 3 ? kp * kp : kp;
  double *o = Q + box * rows * kp + (int64_t)r * kp;
#pragma unroll
  for (int t = 0; t < KP; ++t)
    if (t < kp && FGT_OK_PTR(o + t)) atomicAdd(o + t, acc[t]);
}

// Targets.  Grid: one CTA per target segment (box b, targets [i0, i1)), one target per thread.  The
// box's incoming grid values are staged through shared memory in slabs of t_d (zero-padded to
// KP x KP per slab; every thread reads the same entry at a time); l_{t_1} lives in registers, l_{t_2}
// and l_{t_3} in shared memory.  The sparse colleagues' sources are then summed directly, and the
// thread writes its target's value.
constexpr size_t kTargetSlabBytes = 64 * 1024;

template <int KP>
__global__ void __launch_bounds__(kPointThreads) point_target_kernel(PointTargets pt, ProxyRule pr, int slab,
                                                                     double *__restrict__ u) {
  extern __shared__ double smt[];
  double *Ls = smt;                                   // [2][KP][kPointThreads]: l_{t_2}, l_{t_3}
  double *Us = smt + 2 * KP * kPointThreads;          // [slab][KP][KP]
  const int d = pt.d, kp = pt.kp, tid = threadIdx.x;
  const int64_t b = pt.tseg[3 * blockIdx.x], i0 = pt.tseg[3 * blockIdx.x + 1], i1 = pt.tseg[3 * blockIdx.x + 2];
  const int in = pt.tbox_in[b];
  const int nq = d == 3 ? kp : 1;                     // slices along t_d
  const int plane = d == 3 ? kp * kp : kp * kp;       // grid values per slice (t_2, t_1)
  for (int64_t base = i0; base < i1; base += kPointThreads) {
    const int64_t i = base + tid;
    const bool live = i < i1;
    double acc = 0.0;
    if (in >= 0) {
      double l1[KP];
#pragma unroll
      for (int t = 0; t < KP; ++t) l1[t] = 0.0;
      if (live) {
        lagrange_reg<KP>(pr, kp, pt.t_local[i * d], l1);
        lagrange_row<KP>(pr, kp, pt.t_local[i * d + 1], Ls + tid, kPointThreads);
        if (d == 3) lagrange_row<KP>(pr, kp, pt.t_local[i * d + 2], Ls + KP * kPointThreads + tid, kPointThreads);
      }
      const double *Ub = pt.U + (int64_t)in * nq * plane;
      for (int s0 = 0; s0 < nq; s0 += slab) {
        const int ns = min(slab, nq - s0);
        __syncthreads();
        for (int e = tid; e < ns * KP * KP; e += kPointThreads) {
          const int q = e / (KP * KP), rem = e - q * KP * KP, r2 = rem / KP, r1 = rem - r2 * KP;
          Us[e] = (r2 < kp && r1 < kp) ? Ub[(int64_t)(s0 + q) * plane + r2 * kp + r1] : 0.0;
        }
        __syncthreads();
        if (!live) continue;
        for (int q = 0; q < ns; ++q) {
          double s2 = 0.0;
          for (int t2 = 0; t2 < kp; ++t2) {
            const double *row = Us + (q * KP + t2) * KP;
            double s1 = 0.0;
#pragma unroll
            for (int t = 0; t < KP; ++t) s1 = fma(l1[t], row[t], s1);
            s2 = fma(Ls[t2 * kPointThreads + tid], s1, s2);
          }
          acc = d == 3 ? fma(Ls[(KP + s0 + q) * kPointThreads + tid], s2, acc) : acc + s2;
        }
      }
    }
    if (!live) continue;
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a) x[a] = pt.t_xyz[i * d + a];
    for (int64_t q = pt.dptr[b]; q < pt.dptr[b + 1]; ++q) {
      const int32_t sb = pt.dbox[q];
      for (int64_t j = pt.sptr[sb]; j < pt.sptr[sb + 1]; ++j) {
        double r2 = 0.0;
        for (int a = 0; a < d; ++a) {
          const double dx = x[a] - __ldg(pt.s_xyz + j * d + a);
          r2 = fma(dx, dx, r2);
        }
        acc = fma(exp(-r2 * pt.inv_delta), __ldg(pt.q_sorted + j), acc);
      }
    }
    if (FGT_OK_PTR(u + pt.t_id[i])) u[pt.t_id[i]] = acc;
  }
}

// ---- FP32 variants (split precision, tol >= 1e-7)

// l_t(s) in FP32 from the normalised barycentric weights: c_t = w_t / (s - x_t) (IEEE reciprocal),
// l_t = c_t / sum_m c_m.  A point within 1e-30 of a node takes that node's unit vector.
template <int KP>
__device__ inline void lagrange_row32(const ProxyRule &pr, int kp, float s, float *l, int stride) {
  float den = 0.f;
  int hit = -1;
  for (int t = 0; t < kp; ++t) {
    const float dx = s - pr.xf[t];
    float c = 0.f;
    if (fabsf(dx) < 1e-30f) hit = t;
    else c = pr.bwf[t] * __frcp_rn(dx);
    l[t * stride] = c;
    den += c;
  }
  for (int t = kp; t < KP; ++t) l[t * stride] = 0.f;
  if (hit >= 0) {
    for (int t = 0; t < kp; ++t) l[t * stride] = (t == hit) ? 1.f : 0.f;
    return;
  }
  const float sc = __frcp_rn(den);
  for (int t = 0; t < kp; ++t) l[t * stride] *= sc;
}

template <int KP>
__device__ inline void lagrange_reg32(const ProxyRule &pr, int kp, float s, float (&l)[KP]) {
  float den = 0.f;
  int hit = -1;
#pragma unroll
  for (int t = 0; t < KP; ++t) {
    l[t] = 0.f;
    if (t < kp) {
      const float dx = s - pr.xf[t];
      if (fabsf(dx) < 1e-30f) hit = t;
      else l[t] = pr.bwf[t] * __frcp_rn(dx);
      den += l[t];
    }
  }
  if (hit >= 0) {
#pragma unroll
    for (int t = 0; t < KP; ++t) l[t] = (t == hit) ? 1.f : 0.f;
    return;
  }
  const float sc = __frcp_rn(den);
#pragma unroll
  for (int t = 0; t < KP; ++t) l[t] *= sc;
}

constexpr int kLChunk32 = 64;  // sources per staged chunk of the FP32 anterpolation

// s + x with the running compensation c (Kahan).
__device__ inline void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// FP32 anterpolation.  Threads form G groups of TG; a thread owns two rows of the block's RB grid rows
// (ra = rt and ra + TG), so every l_{t_1} pair read from shared memory feeds four FMAs.  A group
// takes every G-th source of a chunk (G = 1 in 3D).  Chunk sums (at most 64 terms) are plain FP32
// and are added into the segment's sums with compensation; the segment's sums go into the box's
// FP64 grid atomically.
template <int KP>
__global__ void __launch_bounds__(256) point_anterp32_kernel(int d, int kp, int RB, int TG, int G, ProxyRule pr,
                                                             const int64_t *__restrict__ seg,
                                                             const double *__restrict__ s_local,
                                                             const double *__restrict__ q_sorted,
                                                             double *__restrict__ Q) {
  static_assert(KP % 2 == 0, "rows are read as float2");
  __shared__ __align__(16) float L[kLChunk32][3][KP];
  __shared__ float qs[kLChunk32];
  const int tid = threadIdx.x, g = tid / TG, rt = tid - g * TG;
  const int rows = d == 3 ? kp * kp : kp;
  const int ra = blockIdx.y * RB + rt, rb = ra + TG;
  const bool act = g < G && rt < RB && ra < rows;
  const bool actb = act && rt + TG < RB && rb < rows;
  const int rbb = actb ? rb : ra;
  const int a2 = ra % kp, a3 = d == 3 ? ra / kp : 0, b2 = rbb % kp, b3 = d == 3 ? rbb / kp : 0;
  const int64_t box = seg[3 * blockIdx.x], j0 = seg[3 * blockIdx.x + 1], j1 = seg[3 * blockIdx.x + 2];
  float acc_a[KP], acc_b[KP], sa[KP], ca[KP], sb[KP], cb[KP];
#pragma unroll
  for (int t = 0; t < KP; ++t) acc_a[t] = acc_b[t] = sa[t] = ca[t] = sb[t] = cb[t] = 0.f;
  for (int64_t c0 = j0; c0 < j1; c0 += kLChunk32) {
    const int nc = (int)min((int64_t)kLChunk32, j1 - c0);
    __syncthreads();
    for (int e = tid; e < nc * d; e += blockDim.x) {
      const int j = e / d, a = e - j * d;
      lagrange_row32<KP>(pr, kp, (float)s_local[(c0 + j) * d + a], &L[j][a][0], 1);
    }
    for (int j = tid; j < nc; j += blockDim.x) qs[j] = (float)q_sorted[c0 + j];
    __syncthreads();
    if (!act) continue;
    for (int j = g; j < nc; j += G) {
      float pa = qs[j] * L[j][1][a2], pb = qs[j] * L[j][1][b2];
      if (d == 3) {
        pa *= L[j][2][a3];
        pb *= L[j][2][b3];
      }
      const float2 *l1 = reinterpret_cast<const float2 *>(&L[j][0][0]);
#pragma unroll
      for (int t = 0; t < KP / 2; ++t) {
        const float2 v = l1[t];
        acc_a[2 * t] = fmaf(pa, v.x, acc_a[2 * t]);
        acc_a[2 * t + 1] = fmaf(pa, v.y, acc_a[2 * t + 1]);
        acc_b[2 * t] = fmaf(pb, v.x, acc_b[2 * t]);
        acc_b[2 * t + 1] = fmaf(pb, v.y, acc_b[2 * t + 1]);
      }
    }
#pragma unroll
    for (int t = 0; t < KP; ++t) {
      kahan_add(sa[t], ca[t], acc_a[t]);
      kahan_add(sb[t], cb[t], acc_b[t]);
      acc_a[t] = acc_b[t] = 0.f;
    }
  }
  if (!act) return;
  double *oa = Q + box * rows * kp + (int64_t)ra * kp;
#pragma unroll
  for (int t = 0; t < KP; ++t)
    if (t < kp && FGT_OK_PTR(oa + t)) atomicAdd(oa + t, (double)sa[t] - (double)ca[t]);
  if (!actb) return;
  double *ob = Q + box * rows * kp + (int64_t)rb * kp;
#pragma unroll
  for (int t = 0; t < KP; ++t)
    if (t < kp && FGT_OK_PTR(ob + t)) atomicAdd(ob + t, (double)sb[t] - (double)cb[t]);
}

// FP32 interpolation to the targets: two targets per thread (base + tid and base + 128 + tid), so
// every grid pair read from shared memory feeds four FMAs.  The box's grid is converted to FP32 in
// shared memory (all of it when it fits, else in slabs of t_d); l_{t_1} of both targets in
// registers, l_{t_2} and l_{t_3} in shared memory.  Sums along t_1 and t_2 are plain FP32 (at most
// 40 terms), the sum along t_3 is compensated.  The direct pairs are summed in FP32 from the local
// coordinates of the target and the source in their boxes (compensated).
template <int KP>
__global__ void __launch_bounds__(kPointThreads) point_target32_kernel(PointTargets pt, ProxyRule pr, int slab,
                                                                       double *__restrict__ u) {
  static_assert(KP % 2 == 0, "rows are read as float2");
  constexpr int NT = 2 * kPointThreads;             // targets per pass
  extern __shared__ float4 smf4[];
  float *Ls = reinterpret_cast<float *>(smf4);       // [2][KP][NT]: l_{t_2}, l_{t_3}
  float *Us = Ls + 2 * KP * NT;                      // [slab][KP][KP]
  const int d = pt.d, kp = pt.kp, tid = threadIdx.x;
  const int64_t b = pt.tseg[3 * blockIdx.x], i0 = pt.tseg[3 * blockIdx.x + 1], i1 = pt.tseg[3 * blockIdx.x + 2];
  const int in = pt.tbox_in[b];
  const int nq = d == 3 ? kp : 1, plane = kp * kp;
  const bool whole = slab >= nq;
  const double *Ub = in >= 0 ? pt.U + (int64_t)in * nq * plane : nullptr;
  auto stage = [&](int s0, int ns) {
    for (int e = tid; e < ns * KP * KP; e += kPointThreads) {
      const int q = e / (KP * KP), rem = e - q * KP * KP, r2 = rem / KP, r1 = rem - r2 * KP;
      Us[e] = (r2 < kp && r1 < kp) ? (float)Ub[(int64_t)(s0 + q) * plane + r2 * kp + r1] : 0.f;
    }
  };
  if (in >= 0 && whole) stage(0, nq);
  for (int64_t base = i0; base < i1; base += NT) {
    const int64_t ia = base + tid, ib = base + kPointThreads + tid;
    const bool la = ia < i1, lb = ib < i1;
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    if (in >= 0) {
      float l1a[KP], l1b[KP];
#pragma unroll
      for (int t = 0; t < KP; ++t) l1a[t] = l1b[t] = 0.f;
      __syncthreads();  // the previous pass is done with Ls
      if (la) {
        lagrange_reg32<KP>(pr, kp, (float)pt.t_local[ia * d], l1a);
        lagrange_row32<KP>(pr, kp, (float)pt.t_local[ia * d + 1], Ls + tid, NT);
        if (d == 3) lagrange_row32<KP>(pr, kp, (float)pt.t_local[ia * d + 2], Ls + KP * NT + tid, NT);
      }
      if (lb) {
        lagrange_reg32<KP>(pr, kp, (float)pt.t_local[ib * d], l1b);
        lagrange_row32<KP>(pr, kp, (float)pt.t_local[ib * d + 1], Ls + kPointThreads + tid, NT);
        if (d == 3) lagrange_row32<KP>(pr, kp, (float)pt.t_local[ib * d + 2], Ls + KP * NT + kPointThreads + tid, NT);
      }
      for (int s0 = 0; s0 < nq; s0 += slab) {
        const int ns = min(slab, nq - s0);
        if (!whole) {
          __syncthreads();
          stage(s0, ns);
        }
        __syncthreads();
        if (!(la || lb)) continue;
        for (int q = 0; q < ns; ++q) {
          float s2a = 0.f, s2b = 0.f;
          for (int t2 = 0; t2 < kp; ++t2) {
            const float2 *row = reinterpret_cast<const float2 *>(Us + (q * KP + t2) * KP);
            float s1a = 0.f, s1b = 0.f, s1c = 0.f, s1d = 0.f;  // even / odd t_1 of both targets
#pragma unroll
            for (int t = 0; t < KP / 2; ++t) {
              const float2 v = row[t];
              s1a = fmaf(l1a[2 * t], v.x, s1a);
              s1b = fmaf(l1b[2 * t], v.x, s1b);
              s1c = fmaf(l1a[2 * t + 1], v.y, s1c);
              s1d = fmaf(l1b[2 * t + 1], v.y, s1d);
            }
            s2a = fmaf(Ls[t2 * NT + tid], s1a + s1c, s2a);
            s2b = fmaf(Ls[t2 * NT + kPointThreads + tid], s1b + s1d, s2b);
          }
          if (d == 3) {
            const int t3 = s0 + q;
            s2a *= Ls[(KP + t3) * NT + tid];
            s2b *= Ls[(KP + t3) * NT + kPointThreads + tid];
          }
          kahan_add(sa, ca, s2a);
          kahan_add(sb, cb, s2b);
        }
      }
    }
    // direct pairs in FP32 from local coordinates (compensated sum), both targets together
    float ta[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < d; ++a) {
      if (la) ta[a] = (float)pt.t_local[ia * d + a];
      if (lb) tb[a] = (float)pt.t_local[ib * d + a];
    }
    float da = 0.f, dca = 0.f, db = 0.f, dcb = 0.f;
    for (int64_t q = pt.dptr[b]; q < pt.dptr[b + 1]; ++q) {
      const int32_t sbx = pt.dbox[q];
      float ba[3] = {0.f, 0.f, 0.f}, bb[3] = {0.f, 0.f, 0.f};
      for (int a = 0, c = pt.dcode[q]; a < d; ++a, c /= 3) {
        const float o2 = 2.f * (float)(c % 3 - 1);
        ba[a] = ta[a] - o2;
        bb[a] = tb[a] - o2;
      }
      for (int64_t j = pt.sptr[sbx]; j < pt.sptr[sbx + 1]; ++j) {
        float ra = 0.f, rb = 0.f;
        for (int a = 0; a < d; ++a) {
          const float y = __ldg(pt.s_local32 + j * d + a);
          ra = fmaf(ba[a] - y, ba[a] - y, ra);
          rb = fmaf(bb[a] - y, bb[a] - y, rb);
        }
        const float qj = __ldg(pt.q32 + j);
        kahan_add(da, dca, qj * expf(-pt.dcoef * ra));
        kahan_add(db, dcb, qj * expf(-pt.dcoef * rb));
      }
    }
    if (la) u[pt.t_id[ia]] = ((double)sa - (double)ca) + ((double)da - (double)dca);
    if (lb) u[pt.t_id[ib]] = ((double)sb - (double)cb) + ((double)db - (double)dcb);
  }
}

__global__ void point_gather_q_kernel(int64_t n, const int64_t *__restrict__ id, const double *__restrict__ q,
                                      double *__restrict__ qs, float *__restrict__ q32) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double v = q[id[j]];
  qs[j] = v;
  if (q32) q32[j] = (float)v;
}

namespace {

template <int KP>
cudaError_t point_anterp_launch(int d, int kp, const ProxyRule &pr, int64_t n_seg, const int64_t *seg,
                                const double *s_local, const double *q_sorted, double *Q, cudaStream_t st) {
  const unsigned ny = d == 3 ? (unsigned)((kp * kp + kPointThreads - 1) / kPointThreads) : 1u;
  point_anterp_kernel<KP><<<dim3((unsigned)n_seg, ny), kPointThreads, 0, st>>>(d, kp, pr, seg, s_local, q_sorted, Q);
  return cudaGetLastError();
}

template <int KP>
cudaError_t point_anterp32_launch(int d, int kp, const ProxyRule &pr, int64_t n_seg, const int64_t *seg,
                                  const double *s_local, const double *q_sorted, double *Q, cudaStream_t st) {
  // 3D: blocks of RB <= 512 grid rows, two rows per thread; 2D: groups of ceil(kp / 2) threads
  const int rows = d == 3 ? kp * kp : kp;
  int RB, TG, G, threads;
  unsigned ny;
  if (d == 3) {
    ny = (unsigned)((rows + 511) / 512);
    RB = (rows + (int)ny - 1) / (int)ny;
    TG = (RB + 1) / 2;
    G = 1;
    threads = (TG + 31) / 32 * 32;
  } else {
    ny = 1;
    RB = kp;
    TG = (kp + 1) / 2;
    threads = 256;
    G = threads / TG;
  }
  point_anterp32_kernel<KP><<<dim3((unsigned)n_seg, ny), threads, 0, st>>>(d, kp, RB, TG, G, pr, seg, s_local,
                                                                            q_sorted, Q);
  return cudaGetLastError();
}

template <int KP>
cudaError_t point_target32_launch(const PointTargets &pt, const ProxyRule &pr, double *u, cudaStream_t st) {
  const size_t slice = sizeof(float) * KP * KP;
  const int nq = pt.d == 3 ? pt.kp : 1;
  const int slab = (int)std::max<size_t>(1, std::min<size_t>((size_t)nq, kTargetSlabBytes / slice));
  const size_t sm = sizeof(float) * 2 * KP * 2 * kPointThreads + slice * slab;
  cudaError_t e = cudaFuncSetAttribute(point_target32_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  point_target32_kernel<KP><<<(unsigned)pt.n_tseg, kPointThreads, sm, st>>>(pt, pr, slab, u);
  return cudaGetLastError();
}

template <int KP>
cudaError_t point_target_launch(const PointTargets &pt, const ProxyRule &pr, double *u, cudaStream_t st) {
  const size_t slice = sizeof(double) * KP * KP;
  const int nq = pt.d == 3 ? pt.kp : 1;
  const int slab = (int)std::max<size_t>(1, std::min<size_t>((size_t)nq, kTargetSlabBytes / slice));
  const size_t sm = sizeof(double) * 2 * KP * kPointThreads + slice * slab;
  cudaError_t e = cudaFuncSetAttribute(point_target_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  point_target_kernel<KP><<<(unsigned)pt.n_tseg, kPointThreads, sm, st>>>(pt, pr, slab, u);
  return cudaGetLastError();
}

// k_p rounded up to an even padded order
#define FGT_KP_SWITCH(kp, CALL)                                                           \
  switch (((kp) + 1) & ~1) {                                                              \
    case 4: return CALL(4); case 6: return CALL(6); case 8: return CALL(8);               \
    case 10: return CALL(10); case 12: return CALL(12); case 14: return CALL(14);         \
    case 16: return CALL(16); case 18: return CALL(18); case 20: return CALL(20);         \
    case 22: return CALL(22); case 24: return CALL(24); case 26: return CALL(26);         \
    case 28: return CALL(28); case 30: return CALL(30); case 32: return CALL(32);         \
    case 34: return CALL(34); case 36: return CALL(36); case 38: return CALL(38);         \
    case 40: return CALL(40);                                                             \
    default: return cudaErrorInvalidValue;                                                \
  }
static_assert(kMaxProxy == 40, "padded proxy orders cover 4..40");
// FP32 kernels: k_p up to kMaxProxy32 (split precision needs tol >= 1e-7, about k_p <= 24)
#define FGT_KP_SWITCH32(kp, CALL)                                                         \
  switch (((kp) + 1) & ~1) {                                                              \
    case 4: return CALL(4); case 6: return CALL(6); case 8: return CALL(8);               \
    case 10: return CALL(10); case 12: return CALL(12); case 14: return CALL(14);         \
    case 16: return CALL(16); case 18: return CALL(18); case 20: return CALL(20);         \
    case 22: return CALL(22); case 24: return CALL(24); case 26: return CALL(26);         \
    case 28: return CALL(28); case 30: return CALL(30);                                   \
    default: return cudaErrorInvalidValue;                                                \
  }
static_assert(kMaxProxy32 == 30, "FP32 padded proxy orders cover 4..30");

}  // namespace

cudaError_t point_anterp(int d, int kp, bool f32, const ProxyRule &pr, int64_t n_dense, int64_t n_seg,
                         const int64_t *seg, const double *s_local, const double *q_sorted, double *Q,
                         cudaStream_t st) {
  if (n_dense <= 0) return cudaSuccess;
  if (kp < 1 || kp > kMaxProxy) return cudaErrorInvalidValue;
  const size_t np = d == 3 ? (size_t)kp * kp * kp : (size_t)kp * kp;
  cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(double) * np * n_dense, st);
  if (e != cudaSuccess || n_seg <= 0) return e;
#define FGT_ANTERP(K) point_anterp_launch<K>(d, kp, pr, n_seg, seg, s_local, q_sorted, Q, st)
#define FGT_ANTERP32(K) point_anterp32_launch<K>(d, kp, pr, n_seg, seg, s_local, q_sorted, Q, st)
  if (f32) {
    FGT_KP_SWITCH32(kp, FGT_ANTERP32)
  }
  FGT_KP_SWITCH(kp, FGT_ANTERP)
#undef FGT_ANTERP32
#undef FGT_ANTERP
}

cudaError_t point_targets(const PointTargets &pt, const ProxyRule &pr, double *u, cudaStream_t st) {
  if (pt.n_tseg <= 0) return cudaSuccess;
  if (pt.kp < 1 || pt.kp > kMaxProxy) return cudaErrorInvalidValue;
#define FGT_TARGETS(K) point_target_launch<K>(pt, pr, u, st)
#define FGT_TARGETS32(K) point_target32_launch<K>(pt, pr, u, st)
  if (pt.f32) {
    FGT_KP_SWITCH32(pt.kp, FGT_TARGETS32)
  }
  FGT_KP_SWITCH(pt.kp, FGT_TARGETS)
#undef FGT_TARGETS32
#undef FGT_TARGETS
}

cudaError_t point_gather_q(int64_t n, const int64_t *s_id, const double *q, double *q_sorted, float *q32,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  point_gather_q_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s_id, q, q_sorted, q32);
  return cudaGetLastError();
}

cudaError_t leaf_errors(int d, int k, int64_t n, const double *vals, double *err, double *sumsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  GLRule gl;
  gl_rule(k, gl.x, gl.w);
  const int np = d == 3 ? k * k * k : k * k;
  const size_t sm = sizeof(double) * (3 * (size_t)np + (size_t)k * k);
  cudaError_t e = cudaFuncSetAttribute(leaf_error_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  leaf_error_kernel<<<(unsigned)n, 256, sm, st>>>(d, k, gl, vals, err, sumsq);
  return cudaGetLastError();
}

cudaError_t merge_children(int d, int k, int64_t n_parents, const int64_t *child_rows, const double *vals,
                           double *parent, cudaStream_t st) {
  if (n_parents <= 0) return cudaSuccess;
  GLRule gl;
  gl_rule(k, gl.x, gl.w);
  const int np = d == 3 ? k * k * k : k * k;
  const size_t sm = sizeof(double) * (2 * (size_t)k * k + 3 * (size_t)np);
  cudaError_t e = cudaFuncSetAttribute(merge_children_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  merge_children_kernel<<<(unsigned)n_parents, 256, sm, st>>>(d, k, gl, child_rows, vals, parent);
  return cudaGetLastError();
}

}  // namespace fgt
