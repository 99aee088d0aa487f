// hf_solve.cu - Krylov solve of the linearised system [A B; C D] d = -R
// (Eq. fully-coupled-fully-discrete) on one GPU.
//
//  * SpMV: thread per element over the structure-of-arrays element-block CSR
//    (coalesced matrix stream, element index fastest), plus the face-node
//    terms of cohesive (alpha) and fluid (beta) facets, plus the pressure rows
//    gathered per pressure unknown.  No atomics: every row has one writer.
//  * Preconditioner: block-Jacobi over subdomains of G consecutive elements
//    (Morton order); inside each subdomain a block ILU(0) of A with element
//    blocks, applied by one CTA per subdomain with a level schedule (levels
//    separated by __syncthreads, elements of a level spread over warps, lane =
//    row).  Pressure rows: block lower-triangular step z_p = S^-1 (r_p - C z_u)
//    with S the diagonal of D - C diag(A)^-1 B taken facet by facet.
//  * GMRES(m), right preconditioned, classical Gram-Schmidt, Givens rotations
//    on device; every reduction is two-level (block partials, last block
//    reduces in fixed order) so results are deterministic.  A cycle of m
//    iterations runs without host synchronisation; kernels after convergence
//    see the done flag and return at once.
//  * Mixed precision: FP32 matrix, factor and Krylov vectors inside FP64
//    iterative refinement (residual and update in FP64).
#include <atomic>
#include <cstddef>
#include <mutex>
#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdio>

#include "hf_internal.h"

namespace hfk {

constexpr int RB = 256;  // threads of reduction kernels

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// ------------------------------------------------------------------ SpMV
// MODE 0: y = J x.  MODE 1 (T = double): y = R(x), the residual.
template <typename T, int DIM, int MODE>
__device__ void add_nl_terms(const DevMesh& m, int e, unsigned nlm, const T* __restrict__ x, T* y) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned;
  unsigned dmask = m.dirmask[e];
  for (int j = 0; j < DIM + 1; ++j) {
    bool al = (nlm >> j) & 1u, be = (nlm >> (4 + j)) & 1u;
    if (!al && !be) continue;
    int f = m.slot_face[j * m.ne + e];
    int s = m.slot_side[j * m.ne + e];
    const double* rec = m.nl + (long long)f * S::nld;
    double n[DIM];
    for (int k = 0; k < DIM; ++k) n[k] = m.fnormal[k * m.nf + f];
    double val[F];
    if (MODE == 0) {
      int em = m.fe[f], ep = m.fe[m.nf + f];
      double jn[F], xp[F];
      for (int b = 0; b < F; ++b) {
        int lm = m.loc_m[b * m.nf + f], lp = m.loc_p[b * m.nf + f];
        double sacc = 0.0;
        for (int k = 0; k < DIM; ++k)
          sacc += n[k] * ((double)x[(long long)ep * NED + lp * DIM + k] - (double)x[(long long)em * NED + lm * DIM + k]);
        jn[b] = sacc;
        int pd = m.fpdof[b * m.nf + f];
        xp[b] = (be && pd >= 0) ? (double)x[m.nu + pd] : 0.0;
      }
      for (int a = 0; a < F; ++a) {
        double v = 0.0;
        for (int b = 0; b < F; ++b) {
          if (al) v += rec[L::Tm + a * F + b] * jn[b];
          if (be) v -= rec[L::Mm + a * F + b] * xp[b];
        }
        val[a] = v;
      }
    } else {
      for (int a = 0; a < F; ++a) val[a] = (al ? rec[L::rc + a] : 0.0) - (be ? rec[L::rp + a] : 0.0);
    }
    double sg = s == 0 ? -1.0 : 1.0;
    for (int a = 0; a < F; ++a) {
      int loc = s == 0 ? m.loc_m[a * m.nf + f] : m.loc_p[a * m.nf + f];
      for (int k = 0; k < DIM; ++k) {
        int row = loc * DIM + k;
        if (!((dmask >> row) & 1u)) y[(long long)e * NED + row] += (T)(sg * n[k] * val[a]);
      }
    }
  }
}

template <typename T, int DIM, int MODE>
__device__ void pressure_row(const DevMesh& m, int g, const T* __restrict__ x, T* __restrict__ y) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned;
  double c = m.scal[0];
  const double fv = m.p_fixval[g];
  if (fv == fv) {  // an essential pressure: identity row p = fv
    y[m.nu + g] = (MODE == 0) ? x[m.nu + g] : (T)((double)x[m.nu + g] - fv);
    return;
  }
  if (!m.p_active[g] || (MODE == 0 && m.phase == 1)) {
    y[m.nu + g] = (MODE == 0) ? x[m.nu + g] : (T)((double)x[m.nu + g] - m.p_v);
    return;
  }
  double acc = 0.0;
  for (int t = m.pinc_ptr[g]; t < m.pinc_ptr[g + 1]; ++t) {
    int f = m.pinc_face[t];
    if (!m.beta[f]) continue;
    int ga = m.pinc_a[t];
    const double* rec = m.nl + (long long)f * S::nld;
    if (MODE == 0) {
      int em = m.fe[f], ep = m.fe[m.nf + f];
      for (int b = 0; b < F; ++b) {
        int lm = m.loc_m[b * m.nf + f], lp = m.loc_p[b * m.nf + f];
        double jn = 0.0;
        for (int k = 0; k < DIM; ++k)
          jn += m.fnormal[k * m.nf + f] *
                ((double)x[(long long)ep * NED + lp * DIM + k] - (double)x[(long long)em * NED + lm * DIM + k]);
        acc += rec[L::Cs + ga * F + b] * jn;
        int pd = m.fpdof[b * m.nf + f];
        acc += rec[L::Dm + ga * F + b] * (double)x[m.nu + pd];
      }
    } else {
      acc += rec[L::rf + ga];
    }
  }
  if (MODE == 1) acc -= m.Q0 * m.inj_w[g];
  y[m.nu + g] = (T)(c * acc);
}

// Node groups: the element's nodes are split into SPMV_P(DIM) groups of two
// nodes; warp g of a CTA owns the 2*DIM rows of group g for 32 consecutive
// elements (lane = element).  Every matrix value is read exactly once, with
// the element index fastest, so each warp load is one contiguous 128/256-byte
// segment.  The group's rows are compile-time, so accumulators stay in
// registers.
template <int DIM> struct SpmvGroups {
  static constexpr int P = Shape<DIM>::nen / 2;   // 3 (2D) or 5 (3D) warps per CTA
  static constexpr int R = 2 * DIM;               // rows per group
};

// facet terms of cohesive (alpha) and fluid (beta) facets for the rows of
// node group GRP only, added into that group's accumulators
template <typename T, int DIM, int MODE, int GRP>
__device__ void add_nl_rows(const DevMesh& m, int e, unsigned nlm, const T* __restrict__ x, T* acc) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned, R = SpmvGroups<DIM>::R;
  unsigned dmask = m.dirmask[e];
  for (int j = 0; j < DIM + 1; ++j) {
    bool al = (nlm >> j) & 1u, be = (nlm >> (4 + j)) & 1u;
    if (!al && !be) continue;
    int f = m.slot_face[j * m.ne + e];
    int s = m.slot_side[j * m.ne + e];
    // face nodes of this facet that belong to the group
    bool any = false;
    for (int a = 0; a < F; ++a) {
      int loc = s == 0 ? m.loc_m[a * m.nf + f] : m.loc_p[a * m.nf + f];
      any |= (loc / 2 == GRP);
    }
    if (!any) continue;
    const double* rec = m.nl + (long long)f * S::nld;
    double n[DIM];
    for (int k = 0; k < DIM; ++k) n[k] = m.fnormal[k * m.nf + f];
    double jn[F], xp[F];
    if (MODE == 0) {
      int em = m.fe[f], ep = m.fe[m.nf + f];
      for (int b = 0; b < F; ++b) {
        int lm = m.loc_m[b * m.nf + f], lp = m.loc_p[b * m.nf + f];
        double sacc = 0.0;
        for (int k = 0; k < DIM; ++k)
          sacc += n[k] * ((double)x[(long long)ep * NED + lp * DIM + k] - (double)x[(long long)em * NED + lm * DIM + k]);
        jn[b] = sacc;
        int pd = m.fpdof[b * m.nf + f];
        xp[b] = (be && pd >= 0) ? (double)x[m.nu + pd] : 0.0;
      }
    }
    double sg = s == 0 ? -1.0 : 1.0;
    for (int a = 0; a < F; ++a) {
      int loc = s == 0 ? m.loc_m[a * m.nf + f] : m.loc_p[a * m.nf + f];
      if (loc / 2 != GRP) continue;
      double v = 0.0;
      if (MODE == 0) {
        for (int b = 0; b < F; ++b) {
          if (al) v += rec[L::Tm + a * F + b] * jn[b];
          if (be) v -= rec[L::Mm + a * F + b] * xp[b];
        }
      } else {
        v = (al ? rec[L::rc + a] : 0.0) - (be ? rec[L::rp + a] : 0.0);
      }
      for (int k = 0; k < DIM; ++k) {
        int row = loc * DIM + k;
        if ((dmask >> row) & 1u) continue;
        int rl = (loc % 2) * DIM + k;
        T add = (T)(sg * n[k] * v);
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (q == rl) acc[q] += add;
      }
    }
  }
}

template <typename T, int DIM, int MODE, int GRP>
__device__ __forceinline__ void spmv_group(const DevMesh& m, const T* __restrict__ dg, const T* __restrict__ off,
                                           const T* __restrict__ x, T* __restrict__ y, int e) {
  using S = Shape<DIM>;
  constexpr int NED = S::ned, NFR = S::nfr, R = SpmvGroups<DIM>::R, R0 = GRP * R;
  const long long ne = m.ne;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = (T)0;
  const T* xe = x + (long long)e * NED;
  const T* dge = dg + e;
#pragma unroll 5
  for (int c = 0; c < NED; ++c) {
    T xc = xe[c];
    const T* col = dge + ((long long)c * NED + R0) * ne;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += ld(col + r * ne) * xc;
  }
#pragma unroll
  for (int j = 0; j < DIM + 1; ++j) {
    int nb = m.nbr[j * ne + e];
    if (nb >= 0) {
      const T* xn = x + (long long)nb * NED;
      const T* ob = off + (long long)j * NED * NFR * ne + e;
#pragma unroll 6
      for (int c = 0; c < NED; ++c) {
        T xc = xn[c];
        const T* col = ob + (long long)c * NFR * ne;
#pragma unroll
        for (int rr = 0; rr < NFR; ++rr) {
          constexpr int dummy = 0;
          (void)dummy;
          const int node = face_node<DIM>(j, rr / DIM);
          if (node / 2 == GRP) acc[(node % 2) * DIM + rr % DIM] += ld(col + rr * ne) * xc;
        }
      }
    }
  }
  unsigned nlm = m.nlmask[e];
  if (nlm) add_nl_rows<T, DIM, MODE, GRP>(m, e, nlm, x, acc);
  T* ye = y + (long long)e * NED + R0;
  if (MODE == 1) {
    unsigned dm = m.dirmask[e];
#pragma unroll
    for (int r = 0; r < R; ++r)
      acc[r] -= (T)(((dm >> (R0 + r)) & 1u) ? m.ubar[(long long)e * NED + R0 + r] : m.fext[(long long)e * NED + R0 + r]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) ye[r] = acc[r];
}

template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(32 * SpmvGroups<DIM>::P, 4) k_spmv(DevMesh m, const T* __restrict__ dg,
                                                                   const T* __restrict__ off, const T* __restrict__ x,
                                                                   T* __restrict__ y, int eblocks, const int* skip) {
  if (skip && *skip) return;
  if ((int)blockIdx.x >= eblocks) {
    int g = (blockIdx.x - eblocks) * blockDim.x + threadIdx.x;
    if (g < m.np) pressure_row<T, DIM, MODE>(m, g, x, y);
    return;
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int e = blockIdx.x * 32 + lane;
  bool live = e < m.ne;
  if (MODE == 0 && m.phase == 2) {
    // fluid-only solve of the staggered scheme: displacement rows are identity
    constexpr int R = SpmvGroups<DIM>::R, NED = Shape<DIM>::ned;
    if (live)
      for (int r = 0; r < R; ++r) y[(long long)e * NED + warp * R + r] = x[(long long)e * NED + warp * R + r];
    return;
  }
  if (live) {
    switch (warp) {
      case 0: spmv_group<T, DIM, MODE, 0>(m, dg, off, x, y, e); break;
      case 1: spmv_group<T, DIM, MODE, 1>(m, dg, off, x, y, e); break;
      case 2: spmv_group<T, DIM, MODE, 2>(m, dg, off, x, y, e); break;
      case 3: if (DIM == 3) spmv_group<T, DIM, MODE, 3>(m, dg, off, x, y, e); break;
      case 4: if (DIM == 3) spmv_group<T, DIM, MODE, 4>(m, dg, off, x, y, e); break;
    }
  }
}

// ------------------------------------------------------------------ ILU(0)
// Row-major scratch per warp: Am (ned x ned) and Lm (nfr x ned).
template <typename T, int DIM>
__device__ void cohesive_patch_rows(const DevMesh& m, int i, int j, int nbside, T* M, int ldm, bool diag,
                                    int lane) {
  // adds alpha * sigma_s sigma_t n_k n_l Tm_ab for the facet of slot j of element i;
  // diag: target is A_ii (rows = element rows); else A_i,nb compact (rows = face rows of slot j)
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn;
  int f = m.slot_face[j * m.ne + i];
  int s = m.slot_side[j * m.ne + i];
  const double* rec = m.nl + (long long)f * S::nld;
  unsigned dmask = m.dirmask[i];
  double sgn = diag ? 1.0 : -1.0;
  for (int t = lane; t < F * F * DIM * DIM; t += 32) {
    int ab = t / (DIM * DIM), kl = t % (DIM * DIM);
    int a = ab / F, b = ab % F, k = kl / DIM, l = kl % DIM;
    int la = s == 0 ? m.loc_m[a * m.nf + f] : m.loc_p[a * m.nf + f];
    int row_el = la * DIM + k;
    if ((dmask >> row_el) & 1u) continue;
    int ts = diag ? s : 1 - s;
    int lb = ts == 0 ? m.loc_m[b * m.nf + f] : m.loc_p[b * m.nf + f];
    int col = lb * DIM + l;
    int row = row_el;
    if (!diag) {
      int fa = 0;
      for (int q = 0; q < F; ++q)
        if (face_node<DIM>(j, q) == la) fa = q;
      row = fa * DIM + k;
    }
    double v = sgn * m.fnormal[k * m.nf + f] * m.fnormal[l * m.nf + f] * rec[L::Tm + a * F + b];
    M[row * ldm + col] += (T)v;
  }
  (void)nbside;
}

template <typename T, int DIM>
__device__ void warp_invert(T* A, int lane) {
  constexpr int N = Shape<DIM>::ned;
  int piv[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // pivot: largest |A[i][k]| for i >= k
    T v = (lane >= k && lane < N) ? (T)fabs((double)A[lane * N + k]) : (T)-1;
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, v, o);
      int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    int p = idx;
    piv[k] = p;
    if (p != k && lane < N) {
      T t = A[k * N + lane];
      A[k * N + lane] = A[p * N + lane];
      A[p * N + lane] = t;
    }
    __syncwarp();
    T pinv = (T)1 / A[k * N + k];
    __syncwarp();
    if (lane < N && lane != k) A[k * N + lane] *= pinv;
    __syncwarp();
    T fk = (lane < N) ? A[lane * N + k] : (T)0;
    __syncwarp();
    if (lane < N && lane != k) {
      for (int c = 0; c < N; ++c)
        if (c != k) A[lane * N + c] -= fk * A[k * N + c];
      A[lane * N + k] = -fk * pinv;
    }
    __syncwarp();
    if (lane == 0) A[k * N + k] = pinv;
    __syncwarp();
  }
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k && lane < N) {
      T t = A[lane * N + k];
      A[lane * N + k] = A[lane * N + p];
      A[lane * N + p] = t;
    }
    __syncwarp();
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_ilu_factor(DevMesh m, const double* __restrict__ dg,
                                                    const double* __restrict__ off, T* lu, const int* sdlist) {
  using S = Shape<DIM>;
  constexpr int NED = S::ned, NFR = S::nfr;
  extern __shared__ __align__(128) unsigned char smraw[];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  T* Am = reinterpret_cast<T*>(smraw) + warp * (NED * NED + NFR * NED);
  T* Lm = Am + NED * NED;
  int s = sdlist[blockIdx.x];
  int lb = m.sd_lvl_base[s], nl = m.sd_nlvl[s];
  const long long ne = m.ne;
  for (int lv = 0; lv < nl; ++lv) {
    int lo = m.sd_lvl[lb + lv], hi = m.sd_lvl[lb + lv + 1];
    for (int idx = lo + warp; idx < hi; idx += nw) {
      int i = m.sd_elems[idx];
      T* recf = lu + m.rec_fwd[i];
      T* recb = lu + m.rec_bwd[i];
      unsigned nlm = m.nlmask[i];
      const unsigned low_i = m.lowmask[i], up_i = m.upmask[i];
      const int nlow_i = nbits(low_i), nup_i = nbits(up_i);
      for (int t = lane; t < NED * NED; t += 32) {
        int r = t / NED, c = t % NED;
        Am[r * NED + c] = (T)dg[((long long)c * NED + r) * ne + i];
      }
      __syncwarp();
      for (int j = 0; j < DIM + 1; ++j) {
        if ((nlm >> j) & 1u) cohesive_patch_rows<T, DIM>(m, i, j, 0, Am, NED, true, lane);
        __syncwarp();
      }
      for (int j = 0; j < DIM + 1; ++j) {
        if (!((low_i >> j) & 1u)) continue;
        int k = m.nbr[j * ne + i];
        // A_ik (compact) into Lm
        for (int t = lane; t < NFR * NED; t += 32) {
          int rr = t / NED, c = t % NED;
          Lm[rr * NED + c] = (T)off[(((long long)j * NED + c) * NFR + rr) * ne + i];
        }
        __syncwarp();
        if ((nlm >> j) & 1u) cohesive_patch_rows<T, DIM>(m, i, j, 1, Lm, NED, false, lane);
        __syncwarp();
        // L_ik = A_ik Dinv_k
        const unsigned up_k = m.upmask[k];
        const T* reckb = lu + m.rec_bwd[k];
        const T* dk = reckb + nbits(up_k) * NED * NFR;
        T lrow[NED];
        if (lane < NFR) {
#pragma unroll
          for (int c = 0; c < NED; ++c) lrow[c] = (T)0;
          for (int mm = 0; mm < NED; ++mm) {
            T a = Lm[lane * NED + mm];
#pragma unroll
            for (int c = 0; c < NED; ++c) lrow[c] += a * dk[c * NED + mm];
          }
        }
        __syncwarp();
        if (lane < NFR) {
#pragma unroll
          for (int c = 0; c < NED; ++c) {
            Lm[lane * NED + c] = lrow[c];
            recf[slots_below(low_i, j) * NED * NFR + c * NFR + lane] = lrow[c];
          }
        }
        __syncwarp();
        // A_ii -= L_ik U_ki, U_ki stored in k's slot that points back to i
        int jk = 0;
        for (int t = 0; t < DIM + 1; ++t)
          if (m.nbr[t * ne + k] == i) jk = t;
        const T* uk = reckb + slots_below(up_k, jk) * NED * NFR;
        for (int t = lane; t < NFR * NED; t += 32) {
          int rr = t / NED, c = t % NED;
          T sacc = (T)0;
          for (int r2 = 0; r2 < NFR; ++r2) {
            int rowk = face_node<DIM>(jk, r2 / DIM) * DIM + r2 % DIM;
            sacc += Lm[rr * NED + rowk] * uk[c * NFR + r2];
          }
          int rowi = face_node<DIM>(j, rr / DIM) * DIM + rr % DIM;
          Am[rowi * NED + c] -= sacc;
        }
        __syncwarp();
      }
      for (int j = 0; j < DIM + 1; ++j) {
        if (!((up_i >> j) & 1u)) continue;
        for (int t = lane; t < NFR * NED; t += 32) {
          int rr = t / NED, c = t % NED;
          Lm[rr * NED + c] = (T)off[(((long long)j * NED + c) * NFR + rr) * ne + i];
        }
        __syncwarp();
        if ((nlm >> j) & 1u) cohesive_patch_rows<T, DIM>(m, i, j, 1, Lm, NED, false, lane);
        __syncwarp();
        for (int t = lane; t < NFR * NED; t += 32) {
          int rr = t / NED, c = t % NED;
          recb[slots_below(up_i, j) * NED * NFR + c * NFR + rr] = Lm[rr * NED + c];
        }
        __syncwarp();
      }
      warp_invert<T, DIM>(Am, lane);
      T* dinv = recb + nup_i * NED * NFR;
      for (int t = lane; t < NED * NED; t += 32) {
        int c = t / NED, r = t % NED;
        dinv[c * NED + r] = Am[r * NED + c];
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

// Schur diagonal of the pressure rows: S = c sum_f [Dm_gg + sum_ab Cs_gb M_ag n.Dinv_(b,a).n]
template <typename T, int DIM>
__global__ void k_schur(DevMesh m, const T* __restrict__ lu, T* sinv) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m.np) return;
  if (!m.p_active[g] || m.p_fixval[g] == m.p_fixval[g]) {
    sinv[g] = (T)1;
    return;
  }
  double c = m.scal[0], sacc = 0.0;
  for (int t = m.pinc_ptr[g]; t < m.pinc_ptr[g + 1]; ++t) {
    int f = m.pinc_face[t];
    if (!m.beta[f]) continue;
    int ga = m.pinc_a[t];
    const double* rec = m.nl + (long long)f * S::nld;
    double n[DIM];
    for (int k = 0; k < DIM; ++k) n[k] = m.fnormal[k * m.nf + f];
    double v = rec[L::Dm + ga * F + ga];
    for (int s = 0; s < 2; ++s) {
      int e = m.fe[s * m.nf + f];
      const T* di = lu + m.rec_bwd[e] + nbits(m.upmask[e]) * NED * S::nfr;
      for (int b = 0; b < F; ++b) {
        int lb = s == 0 ? m.loc_m[b * m.nf + f] : m.loc_p[b * m.nf + f];
        double cs = rec[L::Cs + ga * F + b];
        for (int a = 0; a < F; ++a) {
          int la = s == 0 ? m.loc_m[a * m.nf + f] : m.loc_p[a * m.nf + f];
          double nd = 0.0;
          for (int l = 0; l < DIM; ++l)
            for (int k = 0; k < DIM; ++k)
              nd += n[l] * (double)di[(la * DIM + k) * NED + (lb * DIM + l)] * n[k];
          v += cs * rec[L::Mm + a * F + ga] * nd;
        }
      }
    }
    sacc += v;
  }
  double Sg = c * sacc;
  if (!(fabs(Sg) > 1e-300)) Sg = 1.0;
  sinv[g] = (T)(1.0 / Sg);
}

// ---- TMA bulk copies and mbarriers (shared-memory staging of ILU records)
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  // order earlier generic-proxy reads of dst before the async-proxy write
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// bounded wait on an mbarrier phase; after `polls` unsuccessful polls raise
// the error flag (the first site to give up: 1 ILU(0) apply, 2-4 the delayed
// CGS2 dot kernel's producer, u/w and consumer waits, 5-6 the update
// kernel's producer and consumer waits, 7 the drain, 8 the self-test) and go on
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned phase, int* err, int polls,
                                          int site = 1) {
  for (int it = 0; it < polls; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (ok) return;
  }
  atomicCAS(err, 0, site);  // the first wait that gave up names its site
}

// z = M^-1 rin on the displacement unknowns.  One warp per subdomain, no
// block-level barriers: the warp solves its subdomain's forward sweep then
// its backward sweep element after element in (reverse) level order.  Its
// factor streams are read front to back through a per-warp ring in shared
// memory, filled by TMA bulk copies up to APPLY_NQ segments ahead of the
// element being solved, so HBM latency is hidden behind the solve.
constexpr int APPLY_NQ = 8;

template <typename T, int DIM> struct ApplyRing {
  static constexpr int BS = Shape<DIM>::ned * Shape<DIM>::nfr;
  static constexpr int SEG = (DIM + 1) * BS + Shape<DIM>::ned * Shape<DIM>::ned;  // largest segment
  static constexpr int RINGV = SEG + BS;                                           // ring capacity (values)
};

template <typename T, int DIM, int W>
__global__ void __launch_bounds__(32 * W) k_ilu_apply(DevMesh m, const T* __restrict__ lu, const T* __restrict__ rin,
                                                      T* z, const int* skip) {
  using S = Shape<DIM>;
  using RGN = ApplyRing<T, DIM>;
  constexpr int NED = S::ned, NFR = S::nfr, BS = RGN::BS, RINGV = RGN::RINGV, NQ = APPLY_NQ;
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-warp region: ring | ys | tmp | queue starts | barriers | task table
  const size_t per_warp =
      ((size_t)(RINGV + m.G * NED + 32) * sizeof(T) + NQ * sizeof(long long) + NQ * 8 + (size_t)m.G * 8 + 127) /
      128 * 128;
  unsigned char* region = smraw + (size_t)warp * per_warp;
  T* ring = reinterpret_cast<T*>(region);
  T* ys = ring + RINGV;
  T* tmp = ys + (size_t)m.G * NED;
  long long* qstart = reinterpret_cast<long long*>(tmp + 32);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(qstart + NQ);
  unsigned char* task = reinterpret_cast<unsigned char*>(bars + NQ);
  if (lane < NQ) mbar_init(&bars[lane], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  const int s = blockIdx.x * W + warp;
  if (s >= m.nsd) return;
  const int base = s * m.G, cnt = min(m.G, m.ne - base);
  for (int t = lane; t < cnt * NED; t += 32) ys[t] = rin[(long long)base * NED + t];
  for (int t = lane; t < cnt * 2; t += 32)
    reinterpret_cast<unsigned*>(task)[t] = reinterpret_cast<const unsigned*>(m.sd_task + (size_t)base * 8)[t];
  // face row of this lane in each facet slot
  int frow[DIM + 1];
#pragma unroll
  for (int j = 0; j < DIM + 1; ++j) frow[j] = face_node<DIM>(j, (lane < NFR ? lane : 0) / DIM) * DIM + lane % DIM;
  __syncwarp();
  unsigned vhead = 0, vtail = 0, qh = 0, qt = 0;

  for (int sweep = 0; sweep < 2; ++sweep) {
    int issue_k = 0;
    const T* src = lu + (sweep == 0 ? m.sd_fwd[s] : m.sd_bwd[s]);  // stream cursor
    auto tk = [&](int k) -> const unsigned char* { return task + 8 * (sweep == 0 ? k : cnt - 1 - k); };
    auto seg_size = [&](const unsigned char* t) -> unsigned {
      return sweep == 0 ? nbits(t[1]) * BS : nbits(t[2]) * BS + NED * NED;
    };
    auto produce = [&]() {
      while (issue_k < cnt && qh - qt < (unsigned)NQ) {
        unsigned sz = seg_size(tk(issue_k));
        if (sz == 0) {
          ++issue_k;
          continue;
        }
        if (qh == qt) {  // nothing in flight: restart at the ring origin
          vhead = (vhead + RINGV - 1) / RINGV * RINGV;
          vtail = vhead;
        }
        unsigned pos = vhead % RINGV;
        unsigned pad = (pos + sz > (unsigned)RINGV) ? RINGV - pos : 0;
        if (vhead + pad + sz - vtail > (unsigned)RINGV) break;  // wait for the consumer to free space
        vhead += pad;
        unsigned start = vhead;
        vhead += sz;
        if (lane == 0) {
          qstart[qh % NQ] = start;
          bulk_load(ring + start % RINGV, src, sz * (unsigned)sizeof(T), &bars[qh % NQ]);
        }
        src += sz;
        ++qh;
        ++issue_k;
      }
      __syncwarp();
    };
    produce();
    for (int k = 0; k < cnt; ++k) {
      const unsigned char* t = tk(k);
      const int li = t[0];
      const unsigned mask = sweep == 0 ? t[1] : t[2];
      const unsigned sz = seg_size(t);
      const T* blk = nullptr;
      if (sz) {
        unsigned q = qt % NQ;
        mbar_wait(&bars[q], (qt / NQ) & 1u, m.err_flag, m.wait_polls);
        blk = ring + (unsigned)qstart[q] % RINGV;
      }
      // all block dot products first (independent), then the row updates in
      // slot order (two facets of an element can share face rows)
      T dj[DIM + 1];
#pragma unroll
      for (int j = 0; j < DIM + 1; ++j) {
        dj[j] = (T)0;
        if (((mask >> j) & 1u) && lane < NFR) {
          const T* bq = blk + slots_below(mask, j) * BS + lane;
          const T* yk = ys + t[4 + j] * NED;
          T d0 = (T)0, d1 = (T)0, d2 = (T)0;
#pragma unroll
          for (int c = 0; c < NED; c += 3) {
            d0 += bq[c * NFR] * yk[c];
            d1 += bq[(c + 1) * NFR] * yk[c + 1];
            d2 += bq[(c + 2) * NFR] * yk[c + 2];
          }
          dj[j] = d0 + d1 + d2;
        }
      }
      T* target = sweep == 0 ? ys + li * NED : tmp;
      if (sweep == 1 && lane < NED) tmp[lane] = ys[li * NED + lane];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < DIM + 1; ++j) {
        if ((mask >> j) & 1u) {
          if (lane < NFR) target[frow[j]] -= dj[j];
          __syncwarp();
        }
      }
      if (sweep == 1) {
        // z_i = Dinv_i (y_i - sum_{upper j} U_ij z_j)
        const T* dinv = blk + nbits(mask) * BS;
        T z0 = (T)0, z1 = (T)0, z2 = (T)0;
        if (lane < NED) {
#pragma unroll
          for (int c = 0; c < NED; c += 3) {
            z0 += dinv[c * NED + lane] * tmp[c];
            z1 += dinv[(c + 1) * NED + lane] * tmp[c + 1];
            z2 += dinv[(c + 2) * NED + lane] * tmp[c + 2];
          }
        }
        __syncwarp();
        if (lane < NED) ys[li * NED + lane] = z0 + z1 + z2;
        __syncwarp();
      }
      if (sz) {
        ++qt;
        vtail = (qt < qh) ? (unsigned)qstart[qt % NQ] : vhead;
      }
      produce();
    }
  }
  for (int t = lane; t < cnt * NED; t += 32) z[(long long)base * NED + t] = ys[t];
}

// pressure part of the preconditioner (after the displacement part)
template <typename T, int DIM>
__global__ void k_prec_p(DevMesh m, const T* __restrict__ rin, const double* scale, T* vout, const T* __restrict__ sinv,
                         T* z, const int* skip) {
  // one warp per pressure row: the lanes share the (incident facet, face
  // node) terms of C z_u, so the row's dependent loads are not serialised
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned;
  if (skip && *skip) return;
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (g >= m.np) return;
  T sc = scale ? (T)(*scale) : (T)1;
  T r = rin[m.nu + g] * sc;
  if (lane == 0 && vout) vout[m.nu + g] = r;
  if (!m.p_active[g] || m.p_fixval[g] == m.p_fixval[g] || m.phase == 1) {
    if (lane == 0) z[m.nu + g] = r;
    return;
  }
  if (m.phase == 2) {
    if (lane == 0) z[m.nu + g] = (T)((double)r * m.sinv_d[g]);
    return;
  }
  const int t0 = m.pinc_ptr[g], nt = (m.pinc_ptr[g + 1] - t0) * F;
  double acc = 0.0;
  for (int q = lane; q < nt; q += 32) {
    const int t = t0 + q / F, b = q % F;
    const int f = m.pinc_face[t];
    if (!m.beta[f]) continue;
    const int ga = m.pinc_a[t];
    const int em = m.fe[f], ep = m.fe[m.nf + f];
    const int lm = m.loc_m[b * m.nf + f], lp = m.loc_p[b * m.nf + f];
    double jn = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      jn += m.fnormal[k * m.nf + f] *
            ((double)z[(long long)ep * NED + lp * DIM + k] - (double)z[(long long)em * NED + lm * DIM + k]);
    acc += m.nl[(long long)f * S::nld + L::Cs + ga * F + b] * jn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) z[m.nu + g] = (T)(((double)r - m.scal[0] * acc) * (double)sinv[g]);
}

// the Arnoldi cycle's done flag, read once per CTA: block 0 of the update
// kernels sets it in the same launch in which the other CTAs read it, and a
// CTA that starts late (other streams' kernels holding the SMs) must not let
// its producer warp and its consumer warps see different values, or the
// consumers wait for copies that are never issued
__device__ __forceinline__ bool cta_done(const GmresState* gs) {
  __shared__ int d;
  if (threadIdx.x == 0) d = *reinterpret_cast<const volatile int*>(&gs->done);
  __syncthreads();
  return d != 0;
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of v into partial[blockIdx.x]; returns true in the last block
// (after all partials are visible), where thread 0 may combine them
__device__ bool block_partial_last(double v, double* partial, int* counter) {
  __shared__ double sm[32];
  __shared__ bool last;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    partial[blockIdx.x] = s;
    __threadfence();
    int t = atomicAdd(counter, 1);
    last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// sum of n partials written by other blocks (visible after their fence and
// the ticket atomic), reduced by the whole block in a fixed order; the result
// is returned to every thread
__device__ double block_sum_partials(const double* partial, int n, int stride, int col) {
  __shared__ double sm[RB / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) s += __ldcg(partial + (long long)b * stride + col);
  s = warp_sum(s);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[warp] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------- Gram-Schmidt
// Classical Gram-Schmidt for Arnoldi step j in three kernels per pass, with
// no serial tail in any of them:
//   k_gs_dot  block partials of V[:, 0..j]^T w (and of ||w||^2);
//   k_gs_sub  every CTA reduces the partial table itself (the same fixed
//             order in every CTA, so all CTAs hold bit-identical
//             coefficients), then w -= V h and block partials of ||w||^2;
//   k_gs_fin  every CTA reduces the norm partials; block 0 applies the Givens
//             rotations to column j (staged in shared memory), all CTAs write
//             v_{j+1} = w / ||w||.  With selective re-orthogonalisation the
//             same kernel instead starts the second pass (its dot products)
//             when the first pass removed more than 1 - eta of ||w||.
// The grid is one CTA per SM (GS_T threads), so a table row holds one
// partial per SM.
constexpr int GS_T = 512;
constexpr int GS_MAXB = GS_MAXB_HOST;  // largest grid the partial tables hold

// reduce-scatter of 32 per-lane values over the warp: afterwards lane l's
// a[0] is the warp sum of a[l] (31 shuffles in a fixed butterfly order)
template <int LEN, typename T> __device__ __forceinline__ void rs_stage(T* a, int lane) {
  const bool up = (lane & LEN) != 0;
#pragma unroll
  for (int k = 0; k < LEN; ++k) {
    const T send = up ? a[k] : a[k + LEN];
    const T keep = up ? a[k + LEN] : a[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, LEN);
  }
}
// 16 per-lane values summed over the warp: afterwards lane l < 16 holds the
// warp sum of a[l] in a[0] (16 + 8 + 4 + 2 + 1 shuffles in a fixed order)
template <typename T> __device__ __forceinline__ T warp_reduce_scatter16(T* a, int lane) {
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], 16);
  rs_stage<8>(a, lane);
  rs_stage<4>(a, lane);
  rs_stage<2>(a, lane);
  rs_stage<1>(a, lane);
  return a[0];
}

// block partials of V[:, 0..j]^T w into part[blockIdx.x * GM_LD + c]; with
// wnorm also of ||w||^2 into column GM_MAX.  Columns go in chunks of 16 (w is
// re-read per chunk, from L2): 16 independent 16-byte loads per thread and
// iteration already keep far more bytes in flight than HBM latency needs.
template <typename T>
__device__ void gs_partial_dots(const T* __restrict__ V, long long ldv, int ncols, const T* __restrict__ w,
                                long long n, double* part, bool wnorm) {
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n, NW = GS_T / 32, CH = 16;
  __shared__ double ws[NW][CH + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  for (int q0 = 0; q0 < ncols; q0 += CH) {
    const int nq = min(CH, ncols - q0);
    const T* Vq = V + (long long)q0 * ldv;
    const bool wn = wnorm && q0 == 0;
    T acc[CH];
    T aw = (T)0;
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = (T)0;
    for (long long iv = tid; iv < nv; iv += stride) {
      const VT wv = reinterpret_cast<const VT*>(w)[iv];
      if (wn) aw += Vec<T>::dot(wv, wv);
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c < nq) acc[c] += Vec<T>::dot(reinterpret_cast<const VT*>(Vq + c * ldv)[iv], wv);
    }
    for (long long i = nv * VN + tid; i < n; i += stride) {
      const T wv = w[i];
      if (wn) aw += wv * wv;
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c < nq) acc[c] += Vq[c * ldv + i] * wv;
    }
    const T col = warp_reduce_scatter16(acc, lane);
    if (lane < CH) ws[warp][lane] = (double)col;
    if (wn) {
      const double s = warp_sum((double)aw);
      if (lane == 0) ws[warp][CH] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < nq || (wn && threadIdx.x == CH)) {
      const int c = threadIdx.x;
      double s = 0.0;
      for (int k = 0; k < NW; ++k) s += ws[k][c];
      part[(long long)blockIdx.x * GM_LD + (c < CH ? q0 + c : GM_MAX)] = s;
    }
    __syncthreads();
  }
}

// sums of the nb block partials of columns cols(v) = v < ncols ? v : GM_MAX
// (v < nvc) into out[], by the whole CTA: thread (group, column) adds the rows
// group, group + groups, ... (independent loads, several in flight), then the
// groups meet in a fixed order
__device__ void gs_reduce_table(const double* part, int nb, int ncols, int nvc, double* out) {
  __shared__ double red[GS_T];
  const int cw = nvc <= 32 ? 32 : nvc <= 64 ? 64 : 128;
  const int groups = GS_T / cw;
  const int c = threadIdx.x % cw, grp = threadIdx.x / cw;
  double s = 0.0;
  if (c < nvc) {
    const int col = c < ncols ? c : GM_MAX;
    int b = grp;
    for (; b + 3 * groups < nb; b += 4 * groups) {
      const double v0 = __ldcg(part + (long long)b * GM_LD + col);
      const double v1 = __ldcg(part + (long long)(b + groups) * GM_LD + col);
      const double v2 = __ldcg(part + (long long)(b + 2 * groups) * GM_LD + col);
      const double v3 = __ldcg(part + (long long)(b + 3 * groups) * GM_LD + col);
      s += v0;
      s += v1;
      s += v2;
      s += v3;
    }
    for (; b < nb; b += groups) s += __ldcg(part + (long long)b * GM_LD + col);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < nvc) {
    double t = 0.0;
    for (int g = 0; g < groups; ++g) t += red[g * cw + threadIdx.x];
    out[threadIdx.x < (unsigned)ncols ? threadIdx.x : GM_MAX] = t;
  }
  __syncthreads();
}

// sum of nb doubles (one per block), the same fixed order in every CTA
__device__ double gs_reduce_vector(const double* p, int nb) {
  __shared__ double sw[GS_T / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += __ldcg(p + b);
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sw[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < GS_T / 32; ++k) t += sw[k];
  __syncthreads();
  return t;
}

template <typename T>
__global__ void __launch_bounds__(GS_T) k_gs_dot(const T* __restrict__ V, long long ldv, int j,
                                                 const T* __restrict__ w, long long n, double* part,
                                                 const GmresState* gs, int wnorm) {
  if (cta_done(gs)) return;
  gs_partial_dots<T>(V, ldv, j + 1, w, n, part, wnorm != 0);
}

// w -= V h with h the reduced first-pass (first = 1, stored into column j of
// H, and ||w||^2 before the pass into gs->nrm2) or second-pass coefficients
// (into gs->h2); block partials of the new ||w||^2 into part2
template <typename T>
__global__ void __launch_bounds__(GS_T) k_gs_sub(const T* __restrict__ V, long long ldv, int j, T* w, long long n,
                                                 const double* part, double* part2, GmresState* gs, int first,
                                                 int wnorm, const int* skipflag) {
  if (cta_done(gs) || (skipflag && *skipflag)) return;
  __shared__ double hs[GM_LD];
  __shared__ T ht[GM_MAX];
  const int ncols = j + 1;
  const int nb = gridDim.x;
  gs_reduce_table(part, nb, ncols, ncols + (first && wnorm ? 1 : 0), hs);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) ht[c] = (T)hs[c];
  if (blockIdx.x == 0) {
    double* dst = first ? gs->H + j * GM_LD : gs->h2;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) dst[c] = hs[c];
    if (first && wnorm && threadIdx.x == 0) gs->nrm2 = hs[GM_MAX];
  }
  __syncthreads();
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  T acc = (T)0;
  for (long long iv = tid; iv < nv; iv += stride) {
    VT ww = reinterpret_cast<const VT*>(w)[iv];
#pragma unroll 8
    for (int c = 0; c < ncols; ++c) Vec<T>::axpy(ww, ht[c], reinterpret_cast<const VT*>(V + c * ldv)[iv]);
    reinterpret_cast<VT*>(w)[iv] = ww;
    acc += Vec<T>::dot(ww, ww);
  }
  for (long long i = nv * VN + tid; i < n; i += stride) {
    T ww = w[i];
    for (int c = 0; c < ncols; ++c) ww -= ht[c] * V[c * ldv + i];
    w[i] = ww;
    acc += ww * ww;
  }
  __shared__ double sw[GS_T / 32];
  const double v = warp_sum((double)acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sw[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < GS_T / 32; ++k) t += sw[k];
    part2[blockIdx.x] = t;
  }
}

// the end of a Gram-Schmidt pass, by mode:
//   0: single pass: finish (Givens on column j, v_{j+1} = w / ||w||);
//   1: second pass: H[:, j] += h2, then finish;
//   2: first of two passes: finish if ||w|| kept at least eta of its length
//      (gs->nrm2 is ||w||^2 before the pass) and set gs->skip2; otherwise
//      clear gs->skip2 and write the second pass's block partials of V^T w
template <typename T>
__global__ void __launch_bounds__(GS_T) k_gs_fin(const T* __restrict__ V_in, T* Vnext, long long ldv, int j,
                                                 const T* __restrict__ w, long long n, const double* part2,
                                                 double* part, GmresState* gs, int mrest, int mode, double eta,
                                                 const int* skipflag) {
  if (cta_done(gs) || (skipflag && *skipflag)) return;
  const int nb = gridDim.x;
  const double nrm2 = gs_reduce_vector(part2, nb);
  const double nrm = sqrt(nrm2);
  bool finish = true;
  if (mode == 2) {
    const double before = sqrt(gs->nrm2);
    finish = nrm >= eta * before || !(before > 0.0);
  }
  if (!finish) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      gs->skip2 = 0;
      gs->reorths += 1;
      gs->reorth_cols += j + 1;
    }
    gs_partial_dots<T>(V_in, ldv, j + 1, w, n, part, false);
    return;
  }
  if (blockIdx.x == 0) {
    __shared__ double hc[GM_LD], csd[GM_MAX], snd[GM_MAX];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      hc[i] = gs->H[j * GM_LD + i] + (mode == 1 ? gs->h2[i] : 0.0);
      if (i < j) {
        csd[i] = gs->cs[i];
        snd[i] = gs->sn[i];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < j; ++i) {
        const double a = hc[i], b = hc[i + 1];
        hc[i] = csd[i] * a + snd[i] * b;
        hc[i + 1] = -snd[i] * a + csd[i] * b;
      }
      const double a = hc[j];
      const double den = hypot(a, nrm);
      const double cs = den > 0.0 ? a / den : 1.0, sn = den > 0.0 ? nrm / den : 0.0;
      hc[j] = den;
      hc[j + 1] = 0.0;
      gs->cs[j] = cs;
      gs->sn[j] = sn;
      const double gj = gs->g[j];
      gs->g[j + 1] = -sn * gj;
      gs->g[j] = cs * gj;
      gs->inv_h = nrm > 0.0 ? 1.0 / nrm : 0.0;
      gs->iters += 1;
      gs->jlast = j + 1;
      if (mode == 2) gs->skip2 = 1;
      if (fabs(gs->g[j + 1]) <= gs->tol_abs || j + 1 >= mrest || !(nrm > 0.0) || !isfinite(nrm)) gs->done = 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) gs->H[j * GM_LD + i] = hc[i];
  }
  // v_{j+1} = w / ||w||: every CTA took the same norm from the same partials
  const T sc = (T)(nrm > 0.0 ? 1.0 / nrm : 0.0);
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  for (long long iv = tid; iv < nv; iv += stride)
    reinterpret_cast<VT*>(Vnext)[iv] = Vec<T>::scale(reinterpret_cast<const VT*>(w)[iv], sc);
  for (long long i = nv * VN + tid; i < n; i += stride) Vnext[i] = w[i] * sc;
}

// ------------------------------------------------------- delayed CGS2 Arnoldi
// Gram-Schmidt with the re-orthogonalisation of each basis vector delayed by
// one Arnoldi step and fused with the next step's projection (the
// low-synchronisation "DCGS2" scheme of Bielich, Langou, Thomas,
// Swirydowicz, Yamazaki and Boman): two sweeps over the basis and one
// global reduction per step, with the orthogonality of two-pass classical
// Gram-Schmidt.
//
// At step j >= 1 the basis holds Q = [v_0 .. v_{j-1}] (final, orthonormal)
// and the lagged vector u_j (projected once, not normalised) in column j;
// w = A M^-1 u_j has been formed.  One reduction gives
//   a = Q^T u_j, b = Q^T w, alpha = u_j.u_j, beta = u_j.w,
// then
//   r = sqrt(alpha - a.a),  v_j = (u_j - Q a) / r              (re-orthogonalised)
//   column j-1 of the Hessenberg matrix H: += a, subdiagonal r   (now final)
//   c = H[0..j, 0..j-1] a  (the Arnoldi relation A M^-1 Q = V H)
//   column j (tentative): h_i = (b_i - c_i) / r (i < j), h_j = ((beta - a.b)/r - c_j)/r
//   u_{j+1} = (w - Q b - d v_j) / r with d = (beta - a.b) / r  (projected once)
// so the sweep needs only a, b, r and d; H and its Givens rotations are kept
// by block 0 alone, which does no sweep.  Step 0 has v_0 final: r = 1, no a.
// The convergence test of column j-1 runs at step j; at the end of a cycle a
// last reduction finalises column m-1.
constexpr int DC_LD = 2 * GM_MAX + 2;  // row length of the reduction table
// The reduction table of the delayed CGS2 step holds values of the Krylov
// type T: the FP32 path adds its partial sums in FP32 all the way to the
// per-CTA rows and across them (one conversion to FP64 per column at the
// end).  Its products already carry FP32 rounding, and FP64 arithmetic runs
// at a small fraction of the FP32 rate on this GPU: per-column FP64 shuffle
// reductions took longer than streaming the column itself.
constexpr int DC_SLAB = 12288;                          // table values staged at a time by dc_reduce
constexpr size_t DC_SMEM = DC_SLAB * sizeof(double);   // 96 KiB of dynamic shared memory (opt-in)

// running sum with its rounding error carried beside it (Knuth's TwoSum:
// s + c equals the exact sum of the added values up to O(eps^2)), for the
// FP32 reductions of the delayed CGS2 step; FP64 sums stay plain (their
// rounding is far below the FP32 products', and FP64 adds are scarce)
template <typename T> struct CSum {
  T s = (T)0, c = (T)0;
  __device__ void add(T v) {
    const T t = s + v, bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ double value() const { return (double)s + (double)c; }
};
template <> struct CSum<double> {
  double s = 0.0;
  __device__ void add(double v) { s += v; }
  __device__ double value() const { return s; }
};

// block partials of [Q^T u, Q^T w, u.u, u.w] (w != null) or [Q^T u, u.u]
template <typename T>
__global__ void __launch_bounds__(GS_T) k_dc_dot(const T* __restrict__ V, long long ldv, int j,
                                                 const T* __restrict__ w, long long n, double* part,
                                                 const GmresState* gs) {
  if (cta_done(gs)) return;
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n, NW = GS_T / 32, CH = sizeof(T) == 4 ? 16 : 8;
  __shared__ T ws[NW][2 * CH + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  const T* u = V + (long long)j * ldv;
  const bool hw = w != nullptr;
  T* row = reinterpret_cast<T*>(part) + (long long)blockIdx.x * DC_LD;
  const int nchunks = j > 0 ? (j + CH - 1) / CH : 1;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int q0 = ch * CH, nq = max(0, min(CH, j - q0));
    const T* Vq = V + (long long)q0 * ldv;
    const bool first = ch == 0;
    T au[CH], aw[CH];
    T uu = (T)0, uw = (T)0;
#pragma unroll
    for (int c = 0; c < CH; ++c) au[c] = aw[c] = (T)0;
    for (long long iv = tid; iv < nv; iv += stride) {
      const VT uv = reinterpret_cast<const VT*>(u)[iv];
      VT wv = Vec<T>::zero();
      if (hw) wv = reinterpret_cast<const VT*>(w)[iv];
      if (first) {
        uu += Vec<T>::dot(uv, uv);
        if (hw) uw += Vec<T>::dot(uv, wv);
      }
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c < nq) {
          const VT q = reinterpret_cast<const VT*>(Vq + c * ldv)[iv];
          au[c] += Vec<T>::dot(q, uv);
          if (hw) aw[c] += Vec<T>::dot(q, wv);
        }
    }
    for (long long i = nv * VN + tid; i < n; i += stride) {
      const T uv = u[i], wv = hw ? w[i] : (T)0;
      if (first) {
        uu += uv * uv;
        uw += uv * wv;
      }
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (c < nq) {
          au[c] += Vq[c * ldv + i] * uv;
          aw[c] += Vq[c * ldv + i] * wv;
        }
    }
    // per warp: lanes c < CH hold column c of both sets
    T su, sw;
    if (CH == 16) {
      su = warp_reduce_scatter16(au, lane);
      sw = hw ? warp_reduce_scatter16(aw, lane) : (T)0;
    } else {
      // 8 columns over 32 lanes: full sums across lane bits 4 and 3, then
      // the reduce-scatter over bits 2..0 leaves column l in lane l (< 8)
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        au[k] += __shfl_xor_sync(0xffffffffu, au[k], 16);
        aw[k] += __shfl_xor_sync(0xffffffffu, aw[k], 16);
      }
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        au[k] += __shfl_xor_sync(0xffffffffu, au[k], 8);
        aw[k] += __shfl_xor_sync(0xffffffffu, aw[k], 8);
      }
      rs_stage<4>(au, lane); rs_stage<2>(au, lane); rs_stage<1>(au, lane);
      rs_stage<4>(aw, lane); rs_stage<2>(aw, lane); rs_stage<1>(aw, lane);
      su = au[0];
      sw = aw[0];
    }
    if (lane < CH) {
      ws[warp][lane] = su;
      ws[warp][CH + lane] = sw;
    }
    if (first) {
      const T a = warp_sum(uu), b = warp_sum(uw);
      if (lane == 0) {
        ws[warp][2 * CH] = a;
        ws[warp][2 * CH + 1] = b;
      }
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 2 * CH + 2) {
      CSum<T> cs;
      for (int k = 0; k < NW; ++k) cs.add(ws[k][t]);
      const T s = (T)cs.value();
      if (t < CH) {
        if (t < nq) row[q0 + t] = s;
      } else if (t < 2 * CH) {
        if (hw && t - CH < nq) row[j + q0 + t - CH] = s;
      } else if (first) {
        if (t == 2 * CH) row[hw ? 2 * j : j] = s;
        else if (hw) row[2 * j + 1] = s;
      }
    }
    __syncthreads();
  }
}

// column sums of the nb x nvc table (row length DC_LD) into out[0..nvc), by
// the whole CTA: the table is staged in shared memory (one slab of up to
// DC_SLAB values at a time, four independent loads per thread and pass),
// then G threads per column add interleaved rows and their G partial sums
// meet in a fixed order: the same order, hence the same result, in every CTA
// (NAMED: run by threads 0 .. GS_T-1 alone, on named barrier 1, while a
// producer warp of the CTA streams; otherwise by the whole CTA)
template <bool NAMED> __device__ __forceinline__ void dc_sync() {
  if (NAMED) asm volatile("bar.sync 1, %0;" ::"n"(GS_T) : "memory");
  else __syncthreads();
}
template <typename RT, bool NAMED = false>
__device__ void dc_reduce(const double* part_raw, int nb, int nvc, double* out, RT* stage) {
  const RT* part = reinterpret_cast<const RT*>(part_raw);
  __shared__ double gpart[GS_T];
  const int rows_per = max(1, DC_SLAB / max(nvc, 1));
  const int nth = NAMED ? GS_T : min((int)blockDim.x, GS_T);  // threads past GS_T only join the barriers
  const int G = max(1, min(8, nth / max(nvc, 1)));
  const int c = threadIdx.x % max(nvc, 1), g = (int)threadIdx.x < nth ? threadIdx.x / max(nvc, 1) : G;
  CSum<RT> acc;
  for (int r0 = 0; r0 < nb; r0 += rows_per) {
    const int nr = min(rows_per, nb - r0);
    const int tot = nr * nvc;
    dc_sync<NAMED>();
    for (int t = threadIdx.x; t < tot; t += 4 * nth) {
      if ((int)threadIdx.x >= nth) break;
      RT v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int tt = t + k * nth;
        v[k] = (RT)0;
        if (tt < tot) {
          const int rr = tt / nvc;
          v[k] = __ldcg(part + (long long)(r0 + rr) * DC_LD + (tt - rr * nvc));
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (t + k * nth < tot) stage[t + k * nth] = v[k];
    }
    dc_sync<NAMED>();
    if (g < G)
      for (int rr = g; rr < nr; rr += G) acc.add(stage[rr * nvc + c]);
  }
  if (g < G) gpart[g * nvc + c] = acc.value();
  dc_sync<NAMED>();
  for (int cc = threadIdx.x; cc < nvc; cc += nth) {
    double t = 0.0;
    for (int k = 0; k < G; ++k) t += gpart[k * nvc + cc];
    out[cc] = t;
  }
  dc_sync<NAMED>();
}

// r = sqrt(u.u - a.a), 1 / r and d = (u.w - a.b) / r of the delayed CGS2
// step, from the reduced table: one warp adds the j products (lanes over k,
// then a fixed butterfly), the block reads the three numbers from shared
// memory.  Every CTA computes them in the same order, hence identically;
// one warp instead of every thread, because FP64 arithmetic is scarce here.
template <bool NAMED = false> __device__ void dc_scalars(const double* red, int j, double* sc) {
  if (threadIdx.x < 32) {
    double ab = 0.0, aa = 0.0;
    for (int k = threadIdx.x; k < j; k += 32) {
      ab += red[k] * red[j + k];
      aa += red[k] * red[k];
    }
    ab = warp_sum(ab);
    aa = warp_sum(aa);
    if (threadIdx.x == 0) {
      const double r2 = red[2 * j] - aa;
      const double r = j == 0 ? 1.0 : (r2 > 0.0 ? sqrt(r2) : 0.0);
      const double inv_r = r > 0.0 ? 1.0 / r : 0.0;
      sc[0] = r;
      sc[1] = inv_r;
      sc[2] = (red[2 * j + 1] - ab) * inv_r;
    }
  }
  dc_sync<NAMED>();
}

// Givens rotations of the final column jc (hc, jc + 2 entries, rotated in
// place) and the convergence test on |g_{jc+1}|, by one block: the earlier
// rotations are staged in shared memory, thread 0 applies them
__device__ void dc_givens_block(GmresState* gs, double* hc, int jc, int mrest) {
  __shared__ double csd[GM_MAX], snd[GM_MAX];
  for (int i = threadIdx.x; i < jc; i += blockDim.x) {
    csd[i] = gs->cs[i];
    snd[i] = gs->sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < jc; ++i) {
      const double a = hc[i], b = hc[i + 1];
      hc[i] = csd[i] * a + snd[i] * b;
      hc[i + 1] = -snd[i] * a + csd[i] * b;
    }
    const double a = hc[jc], sub = hc[jc + 1];
    const double den = hypot(a, sub);
    const double cs = den > 0.0 ? a / den : 1.0, sn = den > 0.0 ? sub / den : 0.0;
    hc[jc] = den;
    hc[jc + 1] = 0.0;
    gs->cs[jc] = cs;
    gs->sn[jc] = sn;
    const double gj = gs->g[jc];
    gs->g[jc + 1] = -sn * gj;
    gs->g[jc] = cs * gj;
    gs->iters = jc + 1;
    gs->jlast = jc + 1;
    if (fabs(gs->g[jc + 1]) <= gs->tol_abs || jc + 1 >= mrest || !(sub > 0.0) || !isfinite(sub)) gs->done = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= jc + 1; i += blockDim.x) gs->H[jc * GM_LD + i] = hc[i];
}

template <typename T>
__global__ void __launch_bounds__(GS_T) k_dc_upd(T* V, long long ldv, int j, const T* __restrict__ w, long long n,
                                                 const double* part, GmresState* gs, int mrest) {
  if (cta_done(gs)) return;
  __shared__ double red[DC_LD];
  __shared__ T coef[2 * GM_MAX];
  __shared__ double hc[GM_LD + 1], cvec[GM_LD];
  const int nb = gridDim.x;
  const int nvc = 2 * j + 2;
  extern __shared__ __align__(16) unsigned char dc_stage[];
  dc_reduce<T>(part, nb, nvc, red, reinterpret_cast<T*>(dc_stage));
  __shared__ double sc[3];
  dc_scalars(red, j, sc);
  const double uw = red[2 * j + 1], r = sc[0], inv_r = sc[1], d = sc[2];
  if (blockIdx.x == 0) {
    // Hessenberg bookkeeping (no sweep in this block)
    if (j == 0) {
      if (threadIdx.x == 0) gs->Hr[0] = uw;
      return;
    }
    double* Hr = gs->Hr;
    for (int i = threadIdx.x; i < j; i += blockDim.x) hc[i] = Hr[(j - 1) * GM_LD + i] + red[i];
    if (threadIdx.x == 0) hc[j] = r;
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) Hr[(j - 1) * GM_LD + i] = hc[i];
    // c = H[0..j, 0..j-1] a with column j-1 from hc: thread (row i, group g)
    // adds columns g, g+4, ... (independent loads), the groups then meet in
    // order
    {
      __shared__ double cpart[4][128];
      const int i = threadIdx.x & 127, g = threadIdx.x >> 7;
      double ci = 0.0;
      if (i <= j) {
#pragma unroll 4
        for (int k = g; k < j - 1; k += 4)
          if (i <= k + 1) ci += Hr[k * GM_LD + i] * red[k];
      }
      cpart[g][i] = ci;
      __syncthreads();
      if (threadIdx.x <= (unsigned)j)
        cvec[threadIdx.x] = ((cpart[0][threadIdx.x] + cpart[1][threadIdx.x]) + (cpart[2][threadIdx.x] +
                            cpart[3][threadIdx.x])) + hc[threadIdx.x] * red[j - 1];
      __syncthreads();
    }
    if (r > 0.0)
      for (int i = threadIdx.x; i <= j; i += blockDim.x)
        Hr[j * GM_LD + i] = i < j ? (red[j + i] - cvec[i]) * inv_r : (d - cvec[j]) * inv_r;
    dc_givens_block(gs, hc, j - 1, mrest);
    return;
  }
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    coef[k] = (T)red[k];
    coef[GM_MAX + k] = (T)red[j + k];
  }
  __syncthreads();
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const T ir = (T)inv_r, dd = (T)d;
  const long long stride = (long long)(gridDim.x - 1) * blockDim.x;
  const long long tid = (blockIdx.x - 1) * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  T* u = V + (long long)j * ldv;
  T* un = V + (long long)(j + 1) * ldv;
  for (long long iv = tid; iv < nv; iv += stride) {
    VT uq = reinterpret_cast<const VT*>(u)[iv];
    VT wq = reinterpret_cast<const VT*>(w)[iv];
#pragma unroll 8
    for (int k = 0; k < j; ++k) {
      const VT q = reinterpret_cast<const VT*>(V + k * ldv)[iv];
      Vec<T>::axpy(uq, coef[k], q);
      Vec<T>::axpy(wq, coef[GM_MAX + k], q);
    }
    const VT vj = Vec<T>::scale(uq, ir);
    Vec<T>::axpy(wq, dd, vj);
    if (j > 0) reinterpret_cast<VT*>(u)[iv] = vj;
    reinterpret_cast<VT*>(un)[iv] = Vec<T>::scale(wq, ir);
  }
  for (long long i = nv * VN + tid; i < n; i += stride) {
    T uq = u[i], wq = w[i];
    for (int k = 0; k < j; ++k) {
      uq -= coef[k] * V[k * ldv + i];
      wq -= coef[GM_MAX + k] * V[k * ldv + i];
    }
    const T vj = uq * ir;
    if (j > 0) u[i] = vj;
    un[i] = (wq - dd * vj) * ir;
  }
}

// ---- the delayed CGS2 with the basis streamed through shared memory
// The register kernels above keep only a batch of loads in flight per
// thread (their accumulators take most of the registers), so each thread
// pays a DRAM round trip every few KB.  These variants stream the basis with
// bulk asynchronous copies (cp.async.bulk) into a ring of row segments in
// shared memory: a producer warp issues the copies up to DCT_S segments ahead,
// waiting for a slot only when the consumers have not yet released it
// (mbarriers, bounded waits), and 16 consumer warps compute from shared
// memory.  The bytes in flight are bounded by shared memory, not registers.
// Each CTA owns a contiguous slice of rb rows (a multiple of 64, so every
// segment starts 256-byte aligned); copies are rounded up to 16 bytes and may
// read up to three elements past n, inside the padded allocations.
constexpr int DCT_CONS = 16;                   // consumer warps
constexpr int DCT_THREADS = 32 * (DCT_CONS + 1);
template <typename T> struct DcTma {
  static constexpr int TR = sizeof(T) == 4 ? 4096 : 2048;  // rows per segment (16 KiB)
  static constexpr int S = sizeof(T) == 4 ? 8 : 5;         // ring slots (128 / 80 KiB in flight)
};

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// barrier over threads 0 .. GS_T-1 of the block (named barrier 1)
__device__ __forceinline__ void sync_gs() { asm volatile("bar.sync 1, %0;" ::"n"(GS_T) : "memory"); }

// after the consumers: wait (bounded) for the last copy issued into each ring
// slot, so that no copy is still in flight when the block exits, even after a
// wait that gave up
__device__ __forceinline__ void dct_drain(unsigned long long* full, int S, long long nseg, int* err, int polls) {
  for (int q = 0; q < S && q < nseg; ++q) {
    const long long last = (nseg - 1 - q) / S;  // the slot's last round
    mbar_wait(&full[q], (unsigned)(last & 1), err, polls, 7);
  }
}

template <typename T> __device__ __forceinline__ unsigned dct_bytes(long long rows) {
  return (unsigned)((rows * (long long)sizeof(T) + 15) / 16 * 16);
}

// block partials of [Q^T u, Q^T w, u.u, u.w] over this CTA's slice, the
// column sums taken column after column: u and w of the slice stay in shared
// memory, the basis columns stream through the ring
template <typename T>
__global__ void __launch_bounds__(DCT_THREADS, 1) k_dc_dot_tma(const T* __restrict__ V, long long ldv, int j,
                                                               const T* __restrict__ w, long long n, double* part,
                                                               const GmresState* gs, long long rb, int polls,
                                                               int* err) {
  if (cta_done(gs)) return;
  constexpr int S = DcTma<T>::S, TR = DcTma<T>::TR, NC = DCT_CONS * 32;
  extern __shared__ __align__(128) unsigned char dsm[];
  T* us = reinterpret_cast<T*>(dsm);
  T* wsl = us + rb;
  T* ring = wsl + rb;
  T* wsum = ring + (size_t)S * TR;  // [DCT_CONS][DC_LD]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(wsum + DCT_CONS * DC_LD);
  unsigned long long* empty = full + S;
  unsigned long long* uwbar = empty + S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)blockIdx.x * rb;
  const long long nr = r0 < n ? (n - r0 < rb ? n - r0 : rb) : 0;
  const int nt = (int)((nr + TR - 1) / TR);
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], DCT_CONS);
    }
    mbar_init(uwbar, (unsigned)max(2 * nt, 1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  const T* u = V + (long long)j * ldv;
  if (warp == DCT_CONS) {
    // producer
    if (lane == 0 && nt > 0) {
      for (int t = 0; t < nt; ++t) {
        const long long a = r0 + (long long)t * TR;
        const unsigned by = dct_bytes<T>(r0 + nr - a < TR ? r0 + nr - a : TR);
        bulk_load(us + (size_t)t * TR, u + a, by, uwbar);
        bulk_load(wsl + (size_t)t * TR, w + a, by, uwbar);
      }
      const long long nseg = (long long)j * nt;
      for (long long k = 0; k < nseg; ++k) {
        const int q = (int)(k % S);
        const long long rnd = k / S;
        if (rnd > 0) mbar_wait(&empty[q], (unsigned)((rnd - 1) & 1), err, polls, 2);
        const int c = (int)(k / nt), t = (int)(k % nt);
        const long long a = r0 + (long long)t * TR;
        bulk_load(ring + (size_t)q * TR, V + (long long)c * ldv + a, dct_bytes<T>(r0 + nr - a < TR ? r0 + nr - a : TR),
                  &full[q]);
      }
    }
  } else {
    // consumers: 16-byte vector loads from shared memory, one accumulator per
    // vector component; a segment shorter than TR (the slice's last tile)
    // takes its whole vectors first, then its last rows one by one
    using VT = typename Vec<T>::type;
    constexpr int VN = Vec<T>::n, VPT = TR / (VN * NC);
    static_assert(TR % (VN * NC) == 0, "a segment splits evenly into the consumers' vectors");
    if (nt > 0) mbar_wait(uwbar, 0u, err, polls, 3);
    {
      VT uu = Vec<T>::zero(), uw = Vec<T>::zero();
      const VT* u4 = reinterpret_cast<const VT*>(us);
      const VT* w4 = reinterpret_cast<const VT*>(wsl);
      const long long nv = nr / VN;
      for (long long i = threadIdx.x; i < nv; i += NC) {
        const VT a = u4[i], b = w4[i];
        Vec<T>::madd(uu, a, a);
        Vec<T>::madd(uw, a, b);
      }
      T su = Vec<T>::hsum(uu), sw = Vec<T>::hsum(uw);
      for (long long l = nv * VN + threadIdx.x; l < nr; l += NC) {
        su += us[l] * us[l];
        sw += us[l] * wsl[l];
      }
      const T a = warp_sum(su), b = warp_sum(sw);
      if (lane == 0) {
        wsum[warp * DC_LD + 2 * j] = a;
        wsum[warp * DC_LD + 2 * j + 1] = b;
      }
    }
    for (int c = 0; c < j; ++c) {
      VT au = Vec<T>::zero(), aw = Vec<T>::zero();
      T tu = (T)0, tw = (T)0;
      for (int t = 0; t < nt; ++t) {
        const long long k = (long long)c * nt + t;
        const int q = (int)(k % S);
        mbar_wait(&full[q], (unsigned)((k / S) & 1), err, polls, 4);
        const T* seg = ring + (size_t)q * TR;
        const T* ut = us + (size_t)t * TR;
        const T* wt = wsl + (size_t)t * TR;
        const VT* seg4 = reinterpret_cast<const VT*>(seg);
        const VT* ut4 = reinterpret_cast<const VT*>(ut);
        const VT* wt4 = reinterpret_cast<const VT*>(wt);
        const int rows = (int)(nr - (long long)t * TR < TR ? nr - (long long)t * TR : TR);
        if (rows == TR) {
#pragma unroll
          for (int e = 0; e < VPT; ++e) {
            const int i = threadIdx.x + e * NC;
            const VT qv = seg4[i];
            Vec<T>::madd(au, qv, ut4[i]);
            Vec<T>::madd(aw, qv, wt4[i]);
          }
        } else {
          const int nv = rows / VN;
          for (int i = threadIdx.x; i < nv; i += NC) {
            const VT qv = seg4[i];
            Vec<T>::madd(au, qv, ut4[i]);
            Vec<T>::madd(aw, qv, wt4[i]);
          }
          for (int l = nv * VN + threadIdx.x; l < rows; l += NC) {
            tu += seg[l] * ut[l];
            tw += seg[l] * wt[l];
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[q]);
      }
      const T a = warp_sum(Vec<T>::hsum(au) + tu), b = warp_sum(Vec<T>::hsum(aw) + tw);
      if (lane == 0) {
        wsum[warp * DC_LD + c] = a;
        wsum[warp * DC_LD + j + c] = b;
      }
    }
    if (warp == 0 && lane == 0) dct_drain(full, S, (long long)j * nt, err, polls);
  }
  __syncthreads();
  T* row = reinterpret_cast<T*>(part) + (long long)blockIdx.x * DC_LD;
  for (int c = threadIdx.x; c < 2 * j + 2; c += blockDim.x) {
    CSum<T> cs;
    for (int k = 0; k < DCT_CONS; ++k) cs.add(wsum[k * DC_LD + c]);
    row[c] = (T)cs.value();
  }
}

// the update sweep of the delayed CGS2 step with the basis streamed through
// the ring, tile after tile: per tile the segments of u_j and w, then of the
// j final basis vectors; each consumer thread keeps its rows' two running
// sums in registers and writes v_j and the next lagged vector at the end of
// the tile.  Block 0 keeps the Hessenberg bookkeeping, as in k_dc_upd; the
// other CTAs share the rows (slices of rb rows).  The producer warp starts
// streaming at once (the copies need nothing from the reduction) while the
// consumer warps reduce the table in a staging area beside the ring, on a
// named barrier of their own.
template <typename T>
__global__ void __launch_bounds__(DCT_THREADS, 1) k_dc_upd_tma(T* V, long long ldv, int j, const T* __restrict__ w,
                                                               long long n, const double* part, GmresState* gs,
                                                               int mrest, long long rb, int polls, int* err) {
  if (cta_done(gs)) return;
  constexpr int S = DcTma<T>::S, TR = DcTma<T>::TR, NC = DCT_CONS * 32;
  __shared__ double red[DC_LD];
  __shared__ T coef[2 * GM_MAX];
  __shared__ double hc[GM_LD + 1], cvec[GM_LD];
  __shared__ __align__(8) unsigned long long full[S], empty[S];
  __shared__ double sc[3];
  extern __shared__ __align__(128) unsigned char dsm[];
  T* ring = reinterpret_cast<T*>(dsm);
  T* stage = ring + (size_t)S * TR;  // dc_reduce's staging area
  const int nb = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)(blockIdx.x - 1) * rb;
  const long long nr = blockIdx.x > 0 && r0 < n ? (n - r0 < rb ? n - r0 : rb) : 0;
  const int nt = (int)((nr + TR - 1) / TR);
  const int per = j + 2;  // segments per tile: u_j, w, Q_0 .. Q_{j-1}
  T* u = V + (long long)j * ldv;
  T* un = V + (long long)(j + 1) * ldv;
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], DCT_CONS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == DCT_CONS) {
    if (lane == 0) {
      const long long nseg = (long long)nt * per;
      for (long long k = 0; k < nseg; ++k) {
        const int q = (int)(k % S);
        const long long rnd = k / S;
        if (rnd > 0) mbar_wait(&empty[q], (unsigned)((rnd - 1) & 1), err, polls, 5);
        const int t = (int)(k / per), m = (int)(k % per);
        const long long a = r0 + (long long)t * TR;
        const T* src = m == 0 ? u + a : m == 1 ? w + a : V + (long long)(m - 2) * ldv + a;
        bulk_load(ring + (size_t)q * TR, src, dct_bytes<T>(r0 + nr - a < TR ? r0 + nr - a : TR), &full[q]);
      }
    }
    return;
  }
  // consumers: threads 0 .. GS_T-1, synchronised on named barrier 1
  dc_reduce<T, true>(part, nb, 2 * j + 2, red, stage);
  dc_scalars<true>(red, j, sc);
  const double uw = red[2 * j + 1], r = sc[0], inv_r = sc[1], d = sc[2];
  if (blockIdx.x == 0) {
    // Hessenberg bookkeeping by the consumer threads (no sweep in this
    // block; its producer issued nothing)
    if (j == 0) {
      if (threadIdx.x == 0) gs->Hr[0] = uw;
      return;
    }
    double* Hr = gs->Hr;
    for (int i = threadIdx.x; i < j; i += GS_T) hc[i] = Hr[(j - 1) * GM_LD + i] + red[i];
    if (threadIdx.x == 0) hc[j] = r;
    sync_gs();
    for (int i = threadIdx.x; i <= j; i += GS_T) Hr[(j - 1) * GM_LD + i] = hc[i];
    {
      __shared__ double cpart[4][128];
      const int i = threadIdx.x & 127, g = threadIdx.x >> 7;
      double ci = 0.0;
      if (i <= j) {
#pragma unroll 4
        for (int k = g; k < j - 1; k += 4)
          if (i <= k + 1) ci += Hr[k * GM_LD + i] * red[k];
      }
      cpart[g][i] = ci;
      sync_gs();
      if (threadIdx.x <= (unsigned)j)
        cvec[threadIdx.x] = ((cpart[0][threadIdx.x] + cpart[1][threadIdx.x]) + (cpart[2][threadIdx.x] +
                            cpart[3][threadIdx.x])) + hc[threadIdx.x] * red[j - 1];
      sync_gs();
    }
    if (r > 0.0)
      for (int i = threadIdx.x; i <= j; i += GS_T)
        Hr[j * GM_LD + i] = i < j ? (red[j + i] - cvec[i]) * inv_r : (d - cvec[j]) * inv_r;
    {
      __shared__ double csd[GM_MAX], snd[GM_MAX];
      const int jc = j - 1;
      for (int i = threadIdx.x; i < jc; i += GS_T) {
        csd[i] = gs->cs[i];
        snd[i] = gs->sn[i];
      }
      sync_gs();
      if (threadIdx.x == 0) {
        for (int i = 0; i < jc; ++i) {
          const double p0 = hc[i], p1 = hc[i + 1];
          hc[i] = csd[i] * p0 + snd[i] * p1;
          hc[i + 1] = -snd[i] * p0 + csd[i] * p1;
        }
        const double a0 = hc[jc], sub = hc[jc + 1];
        const double den = hypot(a0, sub);
        const double cs = den > 0.0 ? a0 / den : 1.0, sn = den > 0.0 ? sub / den : 0.0;
        hc[jc] = den;
        hc[jc + 1] = 0.0;
        gs->cs[jc] = cs;
        gs->sn[jc] = sn;
        const double gj = gs->g[jc];
        gs->g[jc + 1] = -sn * gj;
        gs->g[jc] = cs * gj;
        gs->iters = jc + 1;
        gs->jlast = jc + 1;
        if (fabs(gs->g[jc + 1]) <= gs->tol_abs || jc + 1 >= mrest || !(sub > 0.0) || !isfinite(sub)) gs->done = 1;
      }
      sync_gs();
      for (int i = threadIdx.x; i <= jc + 1; i += GS_T) gs->H[jc * GM_LD + i] = hc[i];
    }
    return;
  }
  for (int k = threadIdx.x; k < j; k += GS_T) {
    coef[k] = (T)red[k];
    coef[GM_MAX + k] = (T)red[j + k];
  }
  sync_gs();
  // each consumer thread owns VPT vectors of every tile; it loads the whole
  // vector even past the slice's last row (the ring slot is TR long, the
  // values there are never stored)
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n, VPT = TR / (VN * NC);
  static_assert(TR % (VN * NC) == 0, "a segment splits evenly into the consumers' vectors");
  const T ir = (T)inv_r, dd = (T)d;
  for (int t = 0; t < nt; ++t) {
    const int rows = (int)(nr - (long long)t * TR < TR ? nr - (long long)t * TR : TR);
    VT su[VPT], sw[VPT];
    for (int m = 0; m < per; ++m) {
      const long long k = (long long)t * per + m;
      const int q = (int)(k % S);
      mbar_wait(&full[q], (unsigned)((k / S) & 1), err, polls, 6);
      const VT* seg = reinterpret_cast<const VT*>(ring + (size_t)q * TR);
      if (m == 0) {
#pragma unroll
        for (int e = 0; e < VPT; ++e) su[e] = seg[threadIdx.x + e * NC];
      } else if (m == 1) {
#pragma unroll
        for (int e = 0; e < VPT; ++e) sw[e] = seg[threadIdx.x + e * NC];
      } else {
        const T cu = coef[m - 2], cw = coef[GM_MAX + m - 2];
#pragma unroll
        for (int e = 0; e < VPT; ++e) {
          const VT v = seg[threadIdx.x + e * NC];
          Vec<T>::axpy(su[e], cu, v);
          Vec<T>::axpy(sw[e], cw, v);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[q]);
    }
    const long long a = r0 + (long long)t * TR;
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int l = (threadIdx.x + e * NC) * VN;
      const VT vj = Vec<T>::scale(su[e], ir);
      VT wn = sw[e];
      Vec<T>::axpy(wn, dd, vj);
      wn = Vec<T>::scale(wn, ir);
      if (l + VN <= rows) {
        if (j > 0) *reinterpret_cast<VT*>(u + a + l) = vj;
        *reinterpret_cast<VT*>(un + a + l) = wn;
      } else if (l < rows) {
        const T* pv = reinterpret_cast<const T*>(&vj);
        const T* pw = reinterpret_cast<const T*>(&wn);
        for (int c = 0; c < VN && l + c < rows; ++c) {
          if (j > 0) u[a + l + c] = pv[c];
          un[a + l + c] = pw[c];
        }
      }
    }
  }
  if (warp == 0 && lane == 0) dct_drain(full, S, (long long)nt * per, err, polls);
}

// end of a cycle that ran all mrest steps: finalise column mrest - 1 from
// the reduction of [Q^T u_m, u_m.u_m]
template <typename T>
__global__ void __launch_bounds__(GS_T) k_dc_close(const double* part, int nb, int m, GmresState* gs) {
  if (cta_done(gs)) return;
  __shared__ double red[DC_LD];
  __shared__ double hc[GM_LD + 1];
  extern __shared__ __align__(16) unsigned char dc_stage[];
  dc_reduce<T>(part, nb, m + 1, red, reinterpret_cast<T*>(dc_stage));
  double aa = 0.0;
  for (int k = 0; k < m; ++k) aa += red[k] * red[k];
  const double r2 = red[m] - aa;
  const double r = r2 > 0.0 ? sqrt(r2) : 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) hc[i] = gs->Hr[(m - 1) * GM_LD + i] + red[i];
  if (threadIdx.x == 0) hc[m] = r;
  __syncthreads();
  for (int i = threadIdx.x; i <= m; i += blockDim.x) gs->Hr[(m - 1) * GM_LD + i] = hc[i];
  __syncthreads();
  dc_givens_block(gs, hc, m - 1, m);
  if (threadIdx.x == 0) gs->done = 1;
}

template <typename T>
__global__ void k_scale_into(const T* __restrict__ w, T* v, long long n, const double* s, const int* skip) {
  if (skip && *skip) return;
  T sc = (T)(*s);
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  for (long long iv = tid; iv < nv; iv += stride)
    reinterpret_cast<VT*>(v)[iv] = Vec<T>::scale(reinterpret_cast<const VT*>(w)[iv], sc);
  for (long long i = nv * VN + tid; i < n; i += stride) v[i] = w[i] * sc;
}

// y = R^-1 g for the rotated Hessenberg matrix of the cycle: the jl x jl
// triangle is staged in shared memory by the whole block, then solved column
// by column (each step one division and a parallel update)
__global__ void __launch_bounds__(256) k_backsolve(GmresState* gs, int mrest) {
  extern __shared__ double Hs[];  // mrest columns of GM_LD, then the right-hand side
  const int jl = gs->jlast;
  double* rhs = Hs + (size_t)mrest * GM_LD;
  for (int t = threadIdx.x; t < jl * GM_LD; t += blockDim.x) Hs[t] = gs->H[t];
  for (int t = threadIdx.x; t < jl; t += blockDim.x) rhs[t] = gs->g[t];
  __syncthreads();
  for (int i = jl - 1; i >= 0; --i) {
    const double d = Hs[i * GM_LD + i];
    const double yi = d != 0.0 ? rhs[i] / d : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) gs->y[i] = yi;
    for (int k = threadIdx.x; k < i; k += blockDim.x) rhs[k] -= Hs[i * GM_LD + k] * yi;
    __syncthreads();
  }
}

template <typename T>
__global__ void k_combine(const T* __restrict__ V, long long ldv, long long n, const GmresState* gs, T* u) {
  __shared__ T y[GM_MAX];
  const int jl = gs->jlast;
  for (int c = threadIdx.x; c < GM_MAX; c += blockDim.x) y[c] = c < jl ? (T)gs->y[c] : (T)0;
  __syncthreads();
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const long long stride = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nv = n / VN;
  for (long long iv = tid; iv < nv; iv += stride) {
    VT s = Vec<T>::zero();
#pragma unroll 8
    for (int c = 0; c < jl; ++c) Vec<T>::fma(s, y[c], reinterpret_cast<const VT*>(V + c * ldv)[iv]);
    reinterpret_cast<VT*>(u)[iv] = s;
  }
  for (long long i = nv * VN + tid; i < n; i += stride) {
    T s = (T)0;
    for (int c = 0; c < jl; ++c) s += y[c] * V[c * ldv + i];
    u[i] = s;
  }
}

template <typename T>
__global__ void k_axpy(T* x, const T* __restrict__ z, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) x[i] += z[i];
}

// r = b - Ax and the start of a GMRES cycle: beta = ||r||, g = beta e1
template <typename T>
__global__ void __launch_bounds__(RB) k_residual_start(const T* __restrict__ b, const T* __restrict__ Ax, T* r, long long n,
                                                       double* partial, int* counter, GmresState* gs, double tol_abs) {
  double acc = 0.0;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    T v = b[i] - (Ax ? Ax[i] : (T)0);
    r[i] = v;
    acc += (double)v * (double)v;
  }
  if (!block_partial_last(acc, partial, counter)) return;
  double b2 = block_sum_partials(partial, gridDim.x, 1, 0);
  if (threadIdx.x == 0) {
    double beta = sqrt(b2);
    gs->beta = beta;
    for (int i = 0; i < GM_LD; ++i) gs->g[i] = 0.0;
    gs->g[0] = beta;
    gs->inv_h = beta > 0.0 ? 1.0 / beta : 0.0;
    gs->tol_abs = tol_abs;
    gs->done = (beta <= tol_abs || !(beta > 0.0)) ? 1 : 0;
    gs->jlast = 0;
    *counter = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(RB) k_norm2(const T* __restrict__ v, long long n, double* partial, int* counter,
                                              double* out) {
  double acc = 0.0;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    acc += (double)v[i] * (double)v[i];
  if (!block_partial_last(acc, partial, counter)) return;
  double tot = block_sum_partials(partial, gridDim.x, 1, 0);
  if (threadIdx.x == 0) {
    *out = tot;
    *counter = 0;
  }
}

// FP64 -> FP32 copy scaled by 1/||r|| (red[0] = ||r||^2)
__global__ void k_demote_scaled(const double* __restrict__ r, float* b, long long n, const double* red) {
  double s = 1.0 / sqrt(*red);
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (float)(r[i] * s);
}
__global__ void k_promote_axpy(double* x, const float* __restrict__ d, long long n, const double* red) {
  double s = sqrt(*red);
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) x[i] += s * (double)d[i];
}
template <typename T>
__global__ void k_fill(T* x, long long n, T v) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) x[i] = v;
}
__global__ void k_d2f(const double* __restrict__ a, float* b, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (float)a[i];
}
__global__ void k_f2d(const float* __restrict__ a, double* b, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (double)a[i];
}
__global__ void k_neg(const double* __restrict__ a, double* b, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = -a[i];
}

// Newton update: X += D, optional cut-off p >= p_v on active pressures, and
// the four squared norms ||dU||, ||U||, ||dP||, ||P|| (out[0..3])
__global__ void __launch_bounds__(RB) k_newton_update(DevMesh m, double* X, const double* __restrict__ Dx,
                                                      double* partial, int* counter, double* out) {
  __shared__ double sm[4][RB / 32];
  __shared__ bool last;
  double a[4] = {0, 0, 0, 0};
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m.N; i += stride) {
    // the increment measured is the change applied to the state, after the
    // pressure cut-off (a clipped pressure that stays clipped has converged)
    const double x0 = X[i];
    double x = x0 + Dx[i];
    bool isp = i >= m.nu;
    if (isp && m.cutoff && m.p_active[i - m.nu] && x < m.p_v) x = m.p_v;
    X[i] = x;
    const double d = x - x0;
    a[isp ? 2 : 0] += d * d;
    a[isp ? 3 : 1] += x * x;
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < 4; ++t) {
    double v = warp_sum(a[t]);
    if (lane == 0) sm[t][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < RB / 32; ++w) s += sm[threadIdx.x][w];
    partial[blockIdx.x * 4 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (last) {
    for (int c = 0; c < 4; ++c) {
      double t = block_sum_partials(partial, gridDim.x, 4, c);
      if (threadIdx.x == 0) out[c] = t;
    }
    if (threadIdx.x == 0) *counter = 0;
  }
}

// fluid-only solves: inverse diagonal of the (scaled) pressure block D
template <int DIM>
__global__ void k_diag_d(DevMesh m) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= m.np) return;
  double dsum = 0.0;
  if (m.p_active[g] && !(m.p_fixval[g] == m.p_fixval[g]))
    for (int t = m.pinc_ptr[g]; t < m.pinc_ptr[g + 1]; ++t) {
      const int f = m.pinc_face[t];
      if (!m.beta[f]) continue;
      const int ga = m.pinc_a[t];
      dsum += m.nl[(long long)f * S::nld + L::Dm + ga * F + ga];
    }
  const double d = m.scal[0] * dsum;
  m.sinv_d[g] = fabs(d) > 1e-300 ? 1.0 / d : 1.0;
}

// b = -R on the rows of one block, zero on the other (staggered scheme):
// keep_u / keep_p select the displacement and pressure rows
__global__ void k_neg_part(const double* __restrict__ R, double* b, long long nu, long long n, int keep_u,
                           int keep_p) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    b[i] = ((i < nu) ? keep_u : keep_p) ? -R[i] : 0.0;
}

template <typename T>
__global__ void k_copy(const T* __restrict__ a, T* b, long long n, const int* skip) {
  if (skip && *skip) return;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = a[i];
}

// The bounded wait of the preconditioner's copy pipeline on an mbarrier that
// nothing completes (one arrival expected, none made): it must give up after
// m.wait_polls polls and raise the error flag.  One thread, no copies issued.
__global__ void k_wait_selftest(DevMesh m) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait(&bar, 0u, m.err_flag, m.wait_polls, 8);
}

// ------------------------------------------------------------------ host side
hf_status set_error(hf_mesh* h, hf_status s, const std::string& msg) {
  h->err = msg;
  return s;
}
hf_status check_cuda(hf_mesh* h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HF_OK;
  h->poisoned = true;
  h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return HF_ERR_CUDA;
}

// ---------------------------------------------------------------- profiling
// Event pairs are recorded only when profiling is on and the GMRES cycle is
// not captured in a graph; elapsed times are read at the next synchronisation.
void prof_begin(hf_mesh* h, int kind) {
  Prof& p = h->prof;
  if (p.capturing) {
    if (p.graph_timing_error) return;
    GraphEv g{kind, p.cap_j, nullptr, nullptr};
    cudaEventCreate(&g.a);
    cudaEventCreate(&g.b);
    cudaEventRecord(g.a, h->stream);
    p.cap_list->push_back(g);
    return;
  }
  if (!p.on) return;
  if (p.n >= PROF_EVENTS) prof_flush(h);
  if (!p.ev[2 * p.n]) {
    cudaEventCreate(&p.ev[2 * p.n]);
    cudaEventCreate(&p.ev[2 * p.n + 1]);
  }
  p.kind[p.n] = kind;
  cudaEventRecord(p.ev[2 * p.n], h->stream);
}
void prof_end(hf_mesh* h) {
  Prof& p = h->prof;
  if (p.capturing) {
    if (!p.graph_timing_error) cudaEventRecord(p.cap_list->back().b, h->stream);
    return;
  }
  if (!p.on) return;
  cudaEventRecord(p.ev[2 * p.n + 1], h->stream);
  p.n += 1;
}
void prof_flush(hf_mesh* h) {
  Prof& p = h->prof;
  if (!p.on || p.n == 0) return;
  cudaEventSynchronize(p.ev[2 * p.n - 1]);
  for (int i = 0; i < p.n; ++i) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]);
    p.ms[p.kind[i]] += ms;
    p.launches[p.kind[i]] += 1;
  }
  p.n = 0;
}

// after a replay of a captured cycle that ran `iters` Arnoldi steps, add the
// durations of the kernels those steps executed
static void prof_flush_graph(hf_mesh* h, const std::vector<GraphEv>& ev, int iters) {
  Prof& p = h->prof;
  if (!p.on) return;
  if (p.graph_timing_error) return;
  for (const GraphEv& g : ev) {
    if (g.j >= iters) continue;
    float ms = 0.0f;
    cudaError_t e = cudaEventElapsedTime(&ms, g.a, g.b);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it so later launch checks stay clean
      p.graph_timing_error = (int)e;
      return;
    }
    p.ms[g.kind] += ms;
    p.launches[g.kind] += 1;
  }
}

static int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T> static T* dalloc(hf_mesh* h, size_t n) {
  return reinterpret_cast<T*>(dev_alloc(h, n * sizeof(T)));
}

// Krylov bases for cycles of up to m vectors (re-allocated when a longer
// cycle is asked for)
hf_status krylov_basis_alloc(hf_mesh* h, int m) {
  m = std::max(1, std::min(GM_MAX, m));
  if (m <= h->m_alloc) return HF_OK;
  const long long ldv = h->K64.ldv;
  dev_free(h, h->K64.V);
  dev_free(h, h->K32.V);
  h->K64.V = dalloc<double>(h, (size_t)ldv * (m + 1));
  h->K32.V = dalloc<float>(h, (size_t)ldv * (m + 1));
  if (!h->K64.V || !h->K32.V) {
    h->m_alloc = 0;
    return set_error(h, HF_ERR_OOM, "device allocation of the Krylov basis failed");
  }
  h->m_alloc = m;
  return HF_OK;
}

// the reduction kernels of the delayed CGS2 stage their table in more than
// the default 48 KiB of shared memory: raise their limit once per process
constexpr int SMEM_OPTIN = 227 * 1024;  // opt-in shared memory per block on this GPU

template <typename T> static void dc_configure() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_dc_upd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DC_SMEM);
    cudaFuncSetAttribute(k_dc_close<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DC_SMEM);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_dc_dot_tma<T>) == cudaSuccess)
      cudaFuncSetAttribute(k_dc_dot_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_OPTIN - (int)fa.sharedSizeBytes);
    if (cudaFuncGetAttributes(&fa, k_dc_upd_tma<T>) == cudaSuccess)
      cudaFuncSetAttribute(k_dc_upd_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_OPTIN - (int)fa.sharedSizeBytes);
    cudaGetLastError();
  });
}

// dynamic shared memory of the streamed delayed CGS2 update kernel: the ring
// and, beside it, the staging area of its table reduction
template <typename T> static size_t dct_upd_smem() {
  return (size_t)DcTma<T>::S * DcTma<T>::TR * sizeof(T) + (size_t)DC_SLAB * sizeof(T);
}

// dynamic shared memory of the streamed delayed CGS2 dot kernel for slices
// of rb rows (u and w of the slice, the ring, the per-warp sums, barriers),
// or 0 when it does not fit beside the kernel's static shared memory
template <typename T> static size_t dct_dot_smem(long long rb) {
  const size_t b = (size_t)2 * rb * sizeof(T) + (size_t)DcTma<T>::S * DcTma<T>::TR * sizeof(T) +
                   (size_t)DCT_CONS * DC_LD * sizeof(T) + (size_t)(2 * DcTma<T>::S + 1) * 8;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k_dc_dot_tma<T>) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b + fa.sharedSizeBytes <= (size_t)SMEM_OPTIN ? b : 0;
}

hf_status solver_alloc(hf_mesh* h) {
  dc_configure<float>();
  dc_configure<double>();
  long long N = h->N;
  int m = std::max(1, std::min(GM_MAX, h->opts.restart));
  long long ldv = (N + 63) / 64 * 64;
  h->red_blocks = 152 * 4;
  h->K64.ldv = ldv;
  h->K32.ldv = ldv;
  h->m_alloc = m;
  h->K64.V = dalloc<double>(h, (size_t)ldv * (m + 1));
  h->K64.w = dalloc<double>(h, N);
  h->K64.z = dalloc<double>(h, N);
  h->K64.u = dalloc<double>(h, N);
  h->K64.x = dalloc<double>(h, N);
  h->K64.b = dalloc<double>(h, N);
  h->K32.V = dalloc<float>(h, (size_t)ldv * (m + 1));
  h->K32.w = dalloc<float>(h, N);
  h->K32.z = dalloc<float>(h, N);
  h->K32.u = dalloc<float>(h, N);
  h->K32.x = dalloc<float>(h, N);
  h->K32.b = dalloc<float>(h, N);
  size_t lus = (size_t)h->ne * (h->dim == 2 ? Shape<2>::lus : Shape<3>::lus);
  h->K64.lu = dalloc<double>(h, lus);
  h->K32.lu = dalloc<float>(h, lus);
  h->K64.sinv = dalloc<double>(h, h->np > 0 ? h->np : 1);
  h->K32.sinv = dalloc<float>(h, h->np > 0 ? h->np : 1);
  size_t nmat = (size_t)h->ne * (h->ned * h->ned + (h->dim + 1) * h->ned * h->nfr);
  h->J32.dg = dalloc<float>(h, nmat);
  h->J32.off = h->J32.dg + (size_t)h->ne * h->ned * h->ned;
  h->d_partial = dalloc<double>(h, std::max((size_t)h->red_blocks * GM_LD, (size_t)GS_MAXB * DC_LD));
  h->d_part2 = dalloc<double>(h, GS_MAXB);
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    h->gs_blocks = std::max(1, std::min(GS_MAXB, sms));
  }
  h->d_gs = dalloc<GmresState>(h, 1);
  if (!h->K64.V || !h->K64.w || !h->K64.z || !h->K64.u || !h->K64.x || !h->K64.b || !h->K32.V ||
      !h->K32.w || !h->K32.z || !h->K32.u || !h->K32.x || !h->K32.b || !h->K64.lu || !h->K32.lu ||
      !h->K64.sinv || !h->K32.sinv || !h->J32.dg || !h->d_partial || !h->d_part2 || !h->d_gs)
    return set_error(h, HF_ERR_OOM, "device allocation of the solver workspace failed");
  cudaMemsetAsync(h->K64.lu, 0, lus * sizeof(double), h->stream);
  cudaMemsetAsync(h->K32.lu, 0, lus * sizeof(float), h->stream);
  cudaMemsetAsync(h->d_gs, 0, sizeof(GmresState), h->stream);
  return HF_OK;
}

void convert_j32(hf_mesh* h) {
  size_t nmat = (size_t)h->ne * (h->ned * h->ned + (h->dim + 1) * h->ned * h->nfr);
  { note_launch(); k_d2f<<<grid_for(nmat, 256, 152 * 16), 256, 0, h->stream>>>(h->J64.dg, h->J32.dg, nmat); }
  h->j32_valid = true;
}

template <int DIM> static size_t factor_smem(int elem_size) {
  using S = Shape<DIM>;
  return (size_t)4 * (S::ned * S::ned + S::nfr * S::ned) * elem_size;
}

template <typename T, int DIM> static void factor_impl(hf_mesh* h, const std::vector<int>& sds, T* lu, T* sinv) {
  if (!sds.empty()) {
    cudaMemcpyAsync(h->d_sdlist, sds.data(), sds.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    size_t sm = factor_smem<DIM>(sizeof(T));
    cudaFuncSetAttribute(k_ilu_factor<T, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    { note_launch(); k_ilu_factor<T, DIM><<<(int)sds.size(), 128, sm, h->stream>>>(h->d, h->J64.dg, h->J64.off, lu, h->d_sdlist); }
  }
  if (h->np > 0) { note_launch(); k_schur<T, DIM><<<(int)((h->np + 127) / 128), 128, 0, h->stream>>>(h->d, lu, sinv); }
}

void factor_subdomains(hf_mesh* h, const std::vector<int>& sds) {
  bool mixed = h->opts.precision == HF_PREC_MIXED;
  prof_begin(h, PK_FACTOR);
  struct End {
    hf_mesh* h;
    ~End() { prof_end(h); }
  } end_{h};
  if (h->dim == 2) {
    if (mixed) factor_impl<float, 2>(h, sds, h->K32.lu, h->K32.sinv);
    else factor_impl<double, 2>(h, sds, h->K64.lu, h->K64.sinv);
  } else {
    if (mixed) factor_impl<float, 3>(h, sds, h->K32.lu, h->K32.sinv);
    else factor_impl<double, 3>(h, sds, h->K64.lu, h->K64.sinv);
  }
}

template <typename T, int DIM, int MODE>
static void spmv(hf_mesh* h, const T* dg, const T* off, const T* x, T* y, const int* skip) {
  constexpr int nt = 32 * SpmvGroups<DIM>::P;
  int eb = (int)((h->ne + 31) / 32);
  int pb = (int)((h->np + nt - 1) / nt);
  { note_launch(); k_spmv<T, DIM, MODE><<<eb + pb, nt, 0, h->stream>>>(h->d, dg, off, x, y, eb, skip); }
}

template <int DIM, typename T> static size_t apply_smem(int G, int W) {
  using S = Shape<DIM>;
  size_t per_warp =
      ((size_t)(ApplyRing<T, DIM>::RINGV + G * S::ned + 32) * sizeof(T) + APPLY_NQ * 8 + APPLY_NQ * 8 + (size_t)G * 8 +
       127) /
      128 * 128;
  return (size_t)W * per_warp;
}

template <typename T, int DIM, int W>
static void launch_apply(hf_mesh* h, const T* lu, const T* rin, T* z, const int* skip) {
  size_t sm = apply_smem<DIM, T>(h->G, W);
  // the opt-in limit only grows, so that handles driven from several host
  // threads never lower it under one another
  static std::atomic<size_t> configured{0};
  static std::mutex raise;
  if (sm > 48 * 1024 && sm > configured.load()) {
    std::lock_guard<std::mutex> lock(raise);
    if (sm > configured.load()) {
      cudaFuncSetAttribute(k_ilu_apply<T, DIM, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      configured.store(sm);
    }
  }
  { note_launch(); k_ilu_apply<T, DIM, W><<<(h->d.nsd + W - 1) / W, 32 * W, sm, h->stream>>>(h->d, lu, rin, z, skip); }
}

template <typename T, int DIM>
static void precond(hf_mesh* h, const Krylov<T>& K, const T* rin, const double* scale, T* vout, T* z,
                    const int* skip) {
  (void)scale;
  (void)vout;
  // warps (subdomains) per CTA: as many as keep at least two CTAs per SM busy
  int nsd = h->d.nsd;
  if (h->d.phase == 2) {
    // fluid-only solve: identity on the displacement rows, diagonal of D on
    // the pressure rows
    { note_launch(); k_copy<T><<<h->red_blocks, RB, 0, h->stream>>>(rin, z, h->nu, skip); }
    if (h->np > 0)
      { note_launch(); k_prec_p<T, DIM><<<(int)((h->np + 7) / 8), 256, 0, h->stream>>>(h->d, rin, nullptr, nullptr, K.sinv, z, skip); }
    return;
  }
  const bool coarse = h->opts.coarse && h->nc > 0;
  // the coarse restriction and solve do not depend on the ILU(0) apply, which
  // keeps only a few warps per SM busy: they run on the side stream beside it
  // (joined before the prolongation).  Event-timed profiling keeps them on
  // the handle's stream so every class is timed alone.
  const bool fork = coarse && h->side && !(h->prof.on && !h->prof.capturing);
  if (coarse) {
    if (fork) {
      cudaEventRecord(h->ev_fork, h->stream);
      cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      coarse_pre<T, DIM>(h, K, rin, skip, h->side);
      cudaEventRecord(h->ev_join, h->side);
    } else {
      prof_begin(h, PK_PREC_AUX);
      coarse_pre<T, DIM>(h, K, rin, skip, h->stream);
      prof_end(h);
    }
  }
  prof_begin(h, PK_PREC);
  if (nsd >= 4 * 2 * 152) launch_apply<T, DIM, 4>(h, K.lu, rin, z, skip);
  else if (nsd >= 2 * 2 * 152) launch_apply<T, DIM, 2>(h, K.lu, rin, z, skip);
  else launch_apply<T, DIM, 1>(h, K.lu, rin, z, skip);
  prof_end(h);
  if (fork) cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  if (coarse || h->np > 0) {
    prof_begin(h, PK_PREC_AUX);
    if (coarse) coarse_post<T, DIM>(h, K, z, skip);
    if (h->np > 0)
      { note_launch(); k_prec_p<T, DIM><<<(int)((h->np + 7) / 8), 256, 0, h->stream>>>(h->d, rin, nullptr, nullptr, K.sinv, z, skip); }
    prof_end(h);
  }
}

// one GMRES(m) cycle on x (V[0] and gs already set by k_residual_start)
template <typename T, int DIM>
static void gmres_cycle(hf_mesh* h, Krylov<T>& K, const T* dg, const T* off, int mrest) {
  GmresState* gs = h->d_gs;
  const int* done = &gs->done;
  long long N = h->N;
  int rb = 2 * 152;
  const int nb = h->gs_blocks;
  for (int j = 0; j < mrest; ++j) {
    T* vj = K.V + (long long)j * K.ldv;
    T* vnext = K.V + (long long)(j + 1) * K.ldv;
    h->prof.cap_j = j;
    precond<T, DIM>(h, K, vj, nullptr, nullptr, K.z, done);
    prof_begin(h, PK_SPMV);
    spmv<T, DIM, 0>(h, dg, off, K.z, K.w, done);
    prof_end(h);
    prof_begin(h, PK_ORTH);
    if (h->opts.reorth == 3) {
      const long long rb_dot = (N + nb - 1) / nb, rb_upd = nb > 1 ? (N + nb - 2) / (nb - 1) : 0;
      const size_t dsm = nb > 1 ? dct_dot_smem<T>((rb_dot + 63) / 64 * 64) : 0;
      if (dsm) {
        // the basis streamed through shared memory by bulk copies
        { note_launch(); k_dc_dot_tma<T><<<nb, DCT_THREADS, dsm, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, gs, (rb_dot + 63) / 64 * 64, h->d.wait_polls, h->d.err_flag); }
        { note_launch(); k_dc_upd_tma<T><<<nb, DCT_THREADS, dct_upd_smem<T>(), h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, gs, mrest, (rb_upd + 63) / 64 * 64, h->d.wait_polls, h->d.err_flag); }
      } else {
        { note_launch(); k_dc_dot<T><<<nb, GS_T, 0, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, gs); }
        { note_launch(); k_dc_upd<T><<<nb, GS_T, DC_SMEM, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, gs, mrest); }
      }
      prof_end(h);
      continue;
    }
    // reorth 1: a second pass only when the first removed more than 30% of
    // ||w|| (the Daniel-Gragg-Kaufman-Stewart test); reorth 2: always
    const bool two = h->opts.reorth > 0;
    const double eta = h->opts.reorth == 2 ? HUGE_VAL : 0.7;
    { note_launch(); k_gs_dot<T><<<nb, GS_T, 0, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, gs, two ? 1 : 0); }
    { note_launch(); k_gs_sub<T><<<nb, GS_T, 0, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, h->d_part2, gs, 1, two ? 1 : 0, nullptr); }
    { note_launch(); k_gs_fin<T><<<nb, GS_T, 0, h->stream>>>(K.V, vnext, K.ldv, j, K.w, N, h->d_part2, h->d_partial, gs, mrest, two ? 2 : 0, eta, nullptr); }
    if (two) {
      { note_launch(); k_gs_sub<T><<<nb, GS_T, 0, h->stream>>>(K.V, K.ldv, j, K.w, N, h->d_partial, h->d_part2, gs, 0, 0, &gs->skip2); }
      { note_launch(); k_gs_fin<T><<<nb, GS_T, 0, h->stream>>>(K.V, vnext, K.ldv, j, K.w, N, h->d_part2, h->d_partial, gs, mrest, 1, eta, &gs->skip2); }
    }
    prof_end(h);
  }
  if (h->opts.reorth == 3) {
    // a cycle that ran all mrest steps still has its last column to finalise
    { note_launch(); k_dc_dot<T><<<nb, GS_T, 0, h->stream>>>(K.V, K.ldv, mrest, nullptr, N, h->d_partial, gs); }
    { note_launch(); k_dc_close<T><<<1, GS_T, DC_SMEM, h->stream>>>(h->d_partial, nb, mrest, gs); }
  }
  {
    const size_t sm = ((size_t)mrest * GM_LD + GM_LD) * sizeof(double);
    static std::atomic<size_t> configured{0};
    static std::mutex raise;
    if (sm > 48 * 1024 && sm > configured.load()) {
      std::lock_guard<std::mutex> lock(raise);
      if (sm > configured.load()) {
        cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        configured.store(sm);
      }
    }
    note_launch();
    k_backsolve<<<1, 256, sm, h->stream>>>(gs, mrest);
  }
  { note_launch(); k_combine<T><<<rb, RB, 0, h->stream>>>(K.V, K.ldv, N, gs, K.u); }
  precond<T, DIM>(h, K, K.u, nullptr, nullptr, K.z, nullptr);
  { note_launch(); k_axpy<T><<<rb, RB, 0, h->stream>>>(K.x, K.z, N); }
}

template <typename T, int DIM>
static hf_status run_cycle_inner(hf_mesh* h, Krylov<T>& K, const T* dg, const T* off, int mrest,
                                 cudaGraphExec_t* gexec, std::vector<GraphEv>* gev);

template <typename T, int DIM>
static hf_status run_cycle(hf_mesh* h, Krylov<T>& K, const T* dg, const T* off, int mrest, cudaGraphExec_t* gexec,
                           std::vector<GraphEv>* gev) {
  Prof& p = h->prof;
  const bool timed = p.cycles && p.cyc_a && p.cyc_b;
  if (timed) cudaEventRecord(p.cyc_a, h->stream);
  hf_status s = run_cycle_inner<T, DIM>(h, K, dg, off, mrest, gexec, gev);
  if (timed) {
    cudaEventRecord(p.cyc_b, h->stream);
    p.cyc_pending = true;
  }
  return s;
}

template <typename T, int DIM>
static hf_status run_cycle_inner(hf_mesh* h, Krylov<T>& K, const T* dg, const T* off, int mrest,
                                 cudaGraphExec_t* gexec, std::vector<GraphEv>* gev) {
  long long& gk = sizeof(T) == 8 ? h->graph_kernels64 : h->graph_kernels32;
  if (!h->opts.use_graphs || h->d.phase != 0) {
    gmres_cycle<T, DIM>(h, K, dg, off, mrest);
    return HF_OK;
  }
  if (!*gexec) {
    for (GraphEv& g : *gev) {
      cudaEventDestroy(g.a);
      cudaEventDestroy(g.b);
    }
    gev->clear();
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return check_cuda(h, e, "cudaStreamBeginCapture");
    h->prof.capturing = true;
    h->prof.cap_list = gev;
    long long before = launch_counter();
    gmres_cycle<T, DIM>(h, K, dg, off, mrest);
    gk = launch_counter() - before;  // kernel nodes of the graph, counted per replay
    launch_counter() = before;
    add_launches(-gk);
    h->prof.capturing = false;
    h->prof.cap_list = nullptr;
    e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return check_cuda(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return check_cuda(h, e, "cudaGraphInstantiate");
  }
  launch_counter() += gk;
  add_launches(gk);
  return check_cuda(h, cudaGraphLaunch(*gexec, h->stream), "cudaGraphLaunch");
}

struct CycleInfo {
  double beta;
  int iters;
  int done;
};

static hf_status read_gs(hf_mesh* h, CycleInfo* ci) {
  GmresState tmp;
  cudaError_t e = cudaMemcpyAsync(&tmp, h->d_gs, offsetof(GmresState, g), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  prof_flush(h);
  if (e != cudaSuccess) return check_cuda(h, e, "gmres state read");
  ci->beta = tmp.beta;
  ci->iters = tmp.iters;
  ci->done = tmp.done;
  h->gs_reorths = tmp.reorths;
  h->gs_reorth_cols = tmp.reorth_cols;
  h->gs_cols += (long long)tmp.iters * (tmp.iters + 1) / 2;
  Prof& p = h->prof;
  if (p.cyc_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.cyc_a, p.cyc_b) == cudaSuccess) {
      p.cycle_ms += ms;
      p.cycle_steps += tmp.iters;
    } else {
      cudaGetLastError();
    }
    p.cyc_pending = false;
  }
  return HF_OK;
}

template <int DIM>
static hf_status solve_impl(hf_mesh* h, const double* b, double* x, hf_newton_report* rep) {
  const hf_solver_opts& o = h->opts;
  long long N = h->N;
  int rb = h->red_blocks;
  int* cnt = h->d_count + 4;
  int mrest = std::max(1, std::min(GM_MAX, std::min(o.restart, h->m_alloc)));
  // ||b||
  { note_launch(); k_norm2<double><<<rb, RB, 0, h->stream>>>(b, N, h->d_partial, cnt, h->d_red); }
  double bn2 = 0.0;
  cudaMemcpyAsync(&bn2, h->d_red, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  hf_status st = check_cuda(h, cudaStreamSynchronize(h->stream), "norm");
  if (st) return st;
  double bnorm = sqrt(bn2);
  if (!std::isfinite(bnorm)) return set_error(h, HF_ERR_NONFINITE, "right-hand side is not finite");
  double tol = o.rtol * bnorm;
  int total = 0, refinements = 0;
  double rnorm = bnorm;
  { note_launch(); k_fill<double><<<rb, RB, 0, h->stream>>>(x, N, 0.0); }
  if (bnorm == 0.0) {
    if (rep) {
      rep->gmres_iters = 0;
      rep->lin_res = 0.0;
      rep->lin_converged = 1;
      rep->refinements = 0;
    }
    return HF_OK;
  }
  // FP32 refinement sweeps first in mixed precision; when two sweeps in a
  // row fail to halve the FP64 residual (an FP32 operator too coarse for this
  // system), the solve goes on in FP64 from the current iterate
  bool use64 = o.precision == HF_PREC_FP64 || h->d.phase != 0, fell_back = false;
  if (!use64) {
    Krylov<float>& K = h->K32;
    if (!h->j32_valid) convert_j32(h);
    double* r = h->r64;
    int poor = 0;
    double prev = bnorm;
    cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    for (;;) {
      { note_launch(); k_norm2<double><<<rb, RB, 0, h->stream>>>(r, N, h->d_partial, cnt, h->d_red); }
      double rn2 = 0.0;
      cudaMemcpyAsync(&rn2, h->d_red, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
      if ((st = check_cuda(h, cudaStreamSynchronize(h->stream), "norm"))) break;
      rnorm = sqrt(rn2);
      if (!std::isfinite(rnorm)) {
        st = set_error(h, HF_ERR_NONFINITE, "refinement residual is not finite");
        break;
      }
      if (rnorm <= tol || total >= o.max_iters) break;
      if (refinements > 0) {
        poor = rnorm > 0.5 * prev ? poor + 1 : 0;
        if (poor >= 2) {
          use64 = fell_back = true;
          break;
        }
      }
      prev = rnorm;
      { note_launch(); k_demote_scaled<<<rb, RB, 0, h->stream>>>(r, K.b, N, h->d_red); }
      { note_launch(); k_fill<float><<<rb, RB, 0, h->stream>>>(K.x, N, 0.0f); }
      // each sweep reduces the residual by inner_rtol, except that a sweep
      // needing less to reach the tolerance asks only for that (with a
      // factor 0.3 of margin for the FP32 operator), so the last sweep does
      // not overshoot the tolerance by orders of magnitude
      const double inner = std::max(o.inner_rtol, std::min(0.5, 0.3 * tol / rnorm));
      // a sweep asked for no reduction (inner tolerance >= 1) runs no cycle
      // and leaves the residual as it is
      int cycle_iters = -1;
      if (inner < 1.0) {
        { note_launch(); k_residual_start<float><<<rb, RB, 0, h->stream>>>(K.b, nullptr, K.V, N, h->d_partial, cnt, h->d_gs, inner); }
        { note_launch(); k_scale_into<float><<<rb, RB, 0, h->stream>>>(K.V, K.V, N, &h->d_gs->inv_h, nullptr); }
        cudaMemsetAsync(&h->d_gs->iters, 0, sizeof(int), h->stream);
        if ((st = run_cycle<float, DIM>(h, K, h->J32.dg, h->J32.off, mrest, &h->graph32, &h->gev32))) break;
        CycleInfo ci;
        if ((st = read_gs(h, &ci))) break;
        if (o.use_graphs) prof_flush_graph(h, h->gev32, ci.iters);
        total += ci.iters;
        cycle_iters = ci.iters;
      }
      refinements += 1;
      { note_launch(); k_promote_axpy<<<rb, RB, 0, h->stream>>>(x, K.x, N, h->d_red); }
      prof_begin(h, PK_SPMV64);
      spmv<double, DIM, 0>(h, h->J64.dg, h->J64.off, x, h->tmp64, nullptr);
      prof_end(h);
      { note_launch(); k_residual_start<double><<<rb, RB, 0, h->stream>>>(b, h->tmp64, r, N, h->d_partial, cnt, h->d_gs + 0, 0.0); }
      if (cycle_iters == 0) break;
    }
  }
  if (use64 && !st) {
    Krylov<double>& K = h->K64;
    if (fell_back) {
      std::vector<int> all(h->d.nsd);
      std::iota(all.begin(), all.end(), 0);
      if (DIM == 2) factor_impl<double, 2>(h, all, h->K64.lu, h->K64.sinv);
      else factor_impl<double, 3>(h, all, h->K64.lu, h->K64.sinv);
      cudaMemcpyAsync(K.x, x, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    } else {
      note_launch();
      k_fill<double><<<rb, RB, 0, h->stream>>>(K.x, N, 0.0);
    }
    // restarted cycles from the true residual; five cycles in a row that each
    // reduce it by less than 1% (stagnation at the attainable accuracy) end
    // the solve
    double prev_cycle = HUGE_VAL;
    int stalled = 0;
    for (;;) {
      spmv<double, DIM, 0>(h, h->J64.dg, h->J64.off, K.x, K.w, nullptr);
      { note_launch(); k_residual_start<double><<<rb, RB, 0, h->stream>>>(b, K.w, K.V, N, h->d_partial, cnt, h->d_gs, tol); }
      { note_launch(); k_scale_into<double><<<rb, RB, 0, h->stream>>>(K.V, K.V, N, &h->d_gs->inv_h, nullptr); }
      CycleInfo ci;
      cudaMemsetAsync(&h->d_gs->iters, 0, sizeof(int), h->stream);
      if ((st = read_gs(h, &ci))) break;
      rnorm = ci.beta;
      if (!std::isfinite(rnorm)) {
        st = set_error(h, HF_ERR_NONFINITE, "GMRES residual is not finite");
        break;
      }
      if (rnorm <= tol || total >= o.max_iters) break;
      stalled = rnorm > 0.99 * prev_cycle ? stalled + 1 : 0;
      if (stalled >= 5) break;
      prev_cycle = rnorm;
      if ((st = run_cycle<double, DIM>(h, K, h->J64.dg, h->J64.off, mrest, &h->graph64, &h->gev64))) break;
      if ((st = read_gs(h, &ci))) break;
      if (o.use_graphs) prof_flush_graph(h, h->gev64, ci.iters);
      total += ci.iters;
    }
    cudaMemcpyAsync(x, K.x, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  }
  if (rep) {
    rep->gmres_iters = total;
    rep->refinements = refinements;
    rep->fp64_fallback = fell_back ? 1 : 0;
    rep->lin_res = rnorm / bnorm;
    rep->lin_converged = rnorm <= tol;
  }
  // a bounded wait inside a kernel that gave up leaves its flag behind
  int flag = 0;
  cudaMemcpyAsync(&flag, h->d.err_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  if (flag) {
    cudaMemsetAsync(h->d.err_flag, 0, sizeof(int), h->stream);
    char msg[96];
    snprintf(msg, sizeof msg, "a bounded device wait timed out in the linear solve (site %d)", flag);
    return set_error(h, HF_ERR_TIMEOUT, msg);
  }
  return st;
}

hf_status linear_solve(hf_mesh* h, const double* b, double* x, hf_newton_report* rep) {
  return h->dim == 2 ? solve_impl<2>(h, b, x, rep) : solve_impl<3>(h, b, x, rep);
}

hf_status residual(hf_mesh* h, const double* X, double* R) {
  prof_begin(h, PK_ASSEMBLY);
  if (h->dim == 2) spmv<double, 2, 1>(h, h->J64.dg, h->J64.off, X, R, nullptr);
  else spmv<double, 3, 1>(h, h->J64.dg, h->J64.off, X, R, nullptr);
  prof_end(h);
  return HF_OK;
}

hf_status apply_jacobian(hf_mesh* h, const double* x, double* y) {
  if (h->dim == 2) spmv<double, 2, 0>(h, h->J64.dg, h->J64.off, x, y, nullptr);
  else spmv<double, 3, 0>(h, h->J64.dg, h->J64.off, x, y, nullptr);
  return HF_OK;
}

double device_norm2(hf_mesh* h, const double* v, long long n) {
  { note_launch(); k_norm2<double><<<h->red_blocks, RB, 0, h->stream>>>(v, n, h->d_partial, h->d_count + 4, h->d_red); }
  double r = 0.0;
  cudaMemcpyAsync(&r, h->d_red, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return r;
}

hf_status newton_update(hf_mesh* h, const double* Dx, double out[4]) {
  prof_begin(h, PK_UPDATE);
  { note_launch(); k_newton_update<<<h->red_blocks, RB, 0, h->stream>>>(h->d, h->X, Dx, h->d_partial, h->d_count + 4, h->d_red); }
  prof_end(h);
  cudaMemcpyAsync(out, h->d_red, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  hf_status s = check_cuda(h, cudaStreamSynchronize(h->stream), "newton update");
  prof_flush(h);
  return s;
}

void launch_neg_part(hf_mesh* h, const double* R, double* b, int keep_u, int keep_p) {
  { note_launch(); k_neg_part<<<h->red_blocks, RB, 0, h->stream>>>(R, b, h->nu, h->N, keep_u, keep_p); }
}

void launch_wait_selftest(hf_mesh* h) {
  note_launch();
  k_wait_selftest<<<1, 32, 0, h->stream>>>(h->d);
}

void launch_diag_d(hf_mesh* h) {
  if (h->np <= 0) return;
  note_launch();
  if (h->dim == 2) k_diag_d<2><<<(int)((h->np + 127) / 128), 128, 0, h->stream>>>(h->d);
  else k_diag_d<3><<<(int)((h->np + 127) / 128), 128, 0, h->stream>>>(h->d);
}

void launch_neg(hf_mesh* h, const double* a, double* b) {
  { note_launch(); k_neg<<<h->red_blocks, RB, 0, h->stream>>>(a, b, h->N); }
}

void launch_precond64(hf_mesh* h, const double* r, double* z) {
  if (h->opts.precision == HF_PREC_MIXED) {
    // the FP32 factor applied to an FP64 vector
    { note_launch(); k_d2f<<<h->red_blocks, RB, 0, h->stream>>>(r, h->K32.b, h->N); }
    if (h->dim == 2) precond<float, 2>(h, h->K32, h->K32.b, nullptr, nullptr, h->K32.z, nullptr);
    else precond<float, 3>(h, h->K32, h->K32.b, nullptr, nullptr, h->K32.z, nullptr);
    { note_launch(); k_f2d<<<h->red_blocks, RB, 0, h->stream>>>(h->K32.z, z, h->N); }
  } else {
    if (h->dim == 2) precond<double, 2>(h, h->K64, r, nullptr, nullptr, z, nullptr);
    else precond<double, 3>(h, h->K64, r, nullptr, nullptr, z, nullptr);
  }
}

}  // namespace hfk
