// hf_coarse.cu - the coarse level of the two-level preconditioner.
//
// One-level block-Jacobi ILU(0) leaves the smooth modes of the elastic
// operator to GMRES: its iteration count grows with the number of
// subdomains and GMRES(m) restarts stall on large meshes.  The coarse space
// here holds the rigid-body modes (translations and infinitesimal rotations)
// of aggregates of consecutive elements (in the internal Morton order),
// zero on Dirichlet rows; the coarse operator is its Galerkin projection
// A0 = Phi^T J_base Phi of the cached linear part of the tangent (bulk and
// intact-facet DG blocks, with the blocks of cracked facets switched off),
// inverted once whenever J_base changes.  The correction is additive:
//   z = M_ILU^-1 r + Phi A0^-1 Phi^T r    on the displacement unknowns,
// applied before the pressure rows of the preconditioner so that they see
// the corrected displacements.
#include <algorithm>
#include <cmath>

#include "hf_internal.h"

namespace hfk {

template <int DIM> __host__ __device__ constexpr int n_modes() { return DIM == 2 ? 3 : 6; }

// value of rigid-body mode `mode` at displacement component `comp` of a node
// with coordinates X (relative to the aggregate centre, scaled by its size):
// translations first, then rotations in the planes (0,1) [, (1,2), (2,0)]
template <int DIM, typename R> __device__ __forceinline__ R rbm(int mode, int comp, const R* X) {
  if (mode < DIM) return comp == mode ? (R)1 : (R)0;
  int q = mode - DIM;
  int a = q, b = (q + 1) % 3;  // rotation in the plane (a, b): u_a = -X_b, u_b = X_a
  if (DIM == 2) {
    a = 0;
    b = 1;
  }
  if (comp == a) return -X[b];
  if (comp == b) return X[a];
  return (R)0;
}

// centre (mean of the vertex coordinates) and size (largest coordinate
// distance of any node from it) of each aggregate; one block per aggregate
template <int DIM> __global__ void k_coarse_geo(DevMesh m, int A, double* geo) {
  __shared__ double red[128][4];
  const int g = blockIdx.x, t = threadIdx.x;
  const int e0 = g * A, e1 = min(m.ne, e0 + A);
  double s[3] = {0, 0, 0};
  for (int e = e0 + t; e < e1; e += 128)
    for (int a = 0; a <= DIM; ++a) {
      int nd = m.enode[(long long)a * m.ne + e];
      for (int k = 0; k < DIM; ++k) s[k] += m.xyz[(long long)nd * DIM + k];
    }
  for (int k = 0; k < 3; ++k) red[t][k] = s[k];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (t < o)
      for (int k = 0; k < 3; ++k) red[t][k] += red[t + o][k];
    __syncthreads();
  }
  double c[3];
  const double cnt = (double)(e1 - e0) * (DIM + 1);
  for (int k = 0; k < 3; ++k) c[k] = red[0][k] / cnt;
  __syncthreads();
  double h = 0.0;
  for (int e = e0 + t; e < e1; e += 128)
    for (int a = 0; a < m.nen; ++a) {
      int nd = m.enode[(long long)a * m.ne + e];
      for (int k = 0; k < DIM; ++k) h = fmax(h, fabs(m.xyz[(long long)nd * DIM + k] - c[k]));
    }
  red[t][0] = h;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (t < o) red[t][0] = fmax(red[t][0], red[t + o][0]);
    __syncthreads();
  }
  if (t < DIM) geo[g * 4 + t] = c[t];
  if (t == 0) geo[g * 4 + 3] = red[0][0] > 0 ? red[0][0] : 1.0;
}

// scaled node coordinates per unknown slot: rc[e*ned + a*DIM + k]
template <int DIM> __global__ void k_coarse_rc(DevMesh m, int A, const double* geo, double* rc64, float* rc32) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)m.ne * m.ned) return;
  int e = (int)(i / m.ned), t = (int)(i % m.ned);
  int a = t / DIM, k = t % DIM, g = e / A;
  int nd = m.enode[(long long)a * m.ne + e];
  double v = (m.xyz[(long long)nd * DIM + k] - geo[g * 4 + k]) / geo[g * 4 + 3];
  rc64[i] = v;
  rc32[i] = (float)v;
}

// A0 = Phi^T J_base Phi, one warp per aggregate (its nm rows of A0, which
// only that warp writes, element after element: the sums are deterministic)
template <int DIM>
__global__ void __launch_bounds__(32) k_coarse_build(DevMesh m, int A, int nc, const double* __restrict__ rc,
                                                     const double* __restrict__ dg, const double* __restrict__ off,
                                                     double* A0) {
  using S = Shape<DIM>;
  constexpr int NED = S::ned, NFR = S::nfr, NM = n_modes<DIM>();
  __shared__ double xs[NED];
  const int g = blockIdx.x, lane = threadIdx.x;
  const int e0 = g * A, e1 = min(m.ne, e0 + A);
  const long long ne = m.ne;
  double acc[NM][NM];
#pragma unroll
  for (int k = 0; k < NM; ++k)
#pragma unroll
    for (int l = 0; l < NM; ++l) acc[k][l] = 0.0;
  for (int e = e0; e < e1; ++e) {
    __syncwarp();
    if (lane < NED) xs[lane] = rc[(long long)e * NED + lane];
    __syncwarp();
    const unsigned dme = m.dirmask[e];
    // diagonal block: lane = column c of J_ee
    if (lane < NED) {
      const int c = lane;
      double u[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) u[k] = 0.0;
      for (int r = 0; r < NED; ++r) {
        if ((dme >> r) & 1u) continue;
        double j = dg[((long long)c * NED + r) * ne + e];
#pragma unroll
        for (int k = 0; k < NM; ++k) u[k] += rbm<DIM>(k, r % DIM, &xs[(r / DIM) * DIM]) * j;
      }
      if (!((dme >> c) & 1u)) {
#pragma unroll
        for (int l = 0; l < NM; ++l) {
          double pc = rbm<DIM>(l, c % DIM, &xs[(c / DIM) * DIM]);
#pragma unroll
          for (int k = 0; k < NM; ++k) acc[k][l] += u[k] * pc;
        }
      }
    }
    // neighbour blocks: rows = face rows of slot j of e, lane = column c of the neighbour
    for (int j = 0; j <= DIM; ++j) {
      const int nb = m.nbr[j * ne + e];
      if (nb < 0) continue;
      const int b = nb / A;
      double pl[NM];
      double u[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) u[k] = 0.0;
      if (lane < NED) {
        const int c = lane;
        const unsigned dmn = m.dirmask[nb];
        double xn[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) xn[k] = rc[(long long)nb * NED + (c / DIM) * DIM + k];
        const bool live = !((dmn >> c) & 1u);
#pragma unroll
        for (int l = 0; l < NM; ++l) pl[l] = live ? rbm<DIM>(l, c % DIM, xn) : 0.0;
        const double* ob = off + ((long long)(j * NED + c) * NFR) * ne + e;
        for (int rr = 0; rr < NFR; ++rr) {
          const int r = face_node<DIM>(j, rr / DIM) * DIM + rr % DIM;
          if ((dme >> r) & 1u) continue;
          double v = ob[(long long)rr * ne];
#pragma unroll
          for (int k = 0; k < NM; ++k) u[k] += rbm<DIM>(k, r % DIM, &xs[(r / DIM) * DIM]) * v;
        }
      } else {
#pragma unroll
        for (int l = 0; l < NM; ++l) pl[l] = 0.0;
      }
      if (b == g) {
#pragma unroll
        for (int k = 0; k < NM; ++k)
#pragma unroll
          for (int l = 0; l < NM; ++l) acc[k][l] += u[k] * pl[l];
      } else {
        // another aggregate's columns: reduce over the lanes now
#pragma unroll
        for (int k = 0; k < NM; ++k)
#pragma unroll
          for (int l = 0; l < NM; ++l) {
            double p = u[k] * pl[l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
            if (lane == 0) A0[(long long)(g * NM + k) * nc + b * NM + l] += p;
          }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NM; ++k)
#pragma unroll
    for (int l = 0; l < NM; ++l) {
      double p = acc[k][l];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == 0) A0[(long long)(g * NM + k) * nc + g * NM + l] += p;
    }
}

// pivot threshold of the elimination: 1e-12 of the largest diagonal entry
__global__ void k_coarse_thresh(const double* A0, int nc, double* thr) {
  __shared__ double red[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < nc; i += 256) v = fmax(v, fabs(A0[(long long)i * nc + i]));
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *thr = 1e-12 * red[0];
}

// Blocked Gauss-Jordan inversion in place, GJB pivots per pass.  The pivots
// are taken in the natural order; a pivot at or below the threshold (a mode
// the linear operator does not constrain, e.g. a piece cut free by cracks)
// drops that mode: its row and column of the result are 0, as if the index
// were deleted from the matrix.  For the pivot set K and the rest R, with
// P = X[K,K]^+ the pivot block inverted by the same elementwise steps:
//   X[K,K] <- P,   X[K,R] <- P X[K,R],   X[R,K] <- -X[R,K] P,
//   X[R,R] <- X[R,R] - X[R,K] P X[K,R].
constexpr int GJB = 32;   // pivots per pass
constexpr int GJT = 64;   // output tile of the update (GJT x GJT per CTA)

// P = X[K,K]^+ by GJB x GJB threads, one element each, the pivots in order
__global__ void __launch_bounds__(GJB * GJB) k_gj_pivot(const double* __restrict__ X, int nc, int k0, int kb,
                                                        const double* __restrict__ thr, double* __restrict__ P) {
  __shared__ double a[GJB][GJB + 1];
  const int l = threadIdx.x / GJB, m = threadIdx.x % GJB;
  const bool in = l < kb && m < kb;
  a[l][m] = in ? X[(long long)(k0 + l) * nc + k0 + m] : 0.0;
  __syncthreads();
  const double t = *thr;
  for (int k = 0; k < kb; ++k) {
    const double p = a[k][k], xik = a[l][k], xkj = a[k][m], xij = a[l][m];
    __syncthreads();
    double out;
    if (!(fabs(p) > t)) {
      out = (l == k || m == k) ? 0.0 : xij;
    } else {
      const double piv = 1.0 / p;
      if (l == k && m == k) out = piv;
      else if (l == k) out = xkj * piv;
      else if (m == k) out = -xik * piv;
      else out = xij - xik * xkj * piv;
    }
    if (in) a[l][m] = out;
    __syncthreads();
  }
  if (in) P[l * GJB + m] = a[l][m];
}

// panel of the pass: W[i,:] = X[i,K] P for rows outside K and -P[i-k0,:] for
// rows inside, one warp per row (lane = column of P); B = X[K,:] copied so
// that the update can overwrite X in place
__global__ void __launch_bounds__(256) k_gj_panel(const double* __restrict__ X, int nc, int k0, int kb,
                                                  const double* __restrict__ P, double* __restrict__ W,
                                                  double* __restrict__ B) {
  __shared__ double ps[GJB][GJB];
  for (int e = threadIdx.x; e < GJB * GJB; e += blockDim.x) ps[e / GJB][e % GJB] = P[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i < nc) {
    double w = 0.0;
    if (i >= k0 && i < k0 + kb) {
      w = lane < kb ? -ps[i - k0][lane] : 0.0;
    } else {
      const double x = lane < kb ? X[(long long)i * nc + k0 + lane] : 0.0;
      for (int l = 0; l < kb; ++l) w += __shfl_sync(0xffffffffu, x, l) * ps[l][lane];
      if (lane >= kb) w = 0.0;
    }
    W[(long long)i * GJB + lane] = w;
  }
  const long long nb = (long long)kb * nc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += (long long)gridDim.x * blockDim.x)
    B[e] = X[(long long)(k0 + e / nc) * nc + e % nc];
}

// the rank-kb update of the pass over GJT x GJT tiles: every element is read
// and written by the thread that owns it, W and B are separate buffers
__global__ void __launch_bounds__(256) k_gj_update(double* __restrict__ X, int nc, int k0, int kb,
                                                   const double* __restrict__ W, const double* __restrict__ B) {
  __shared__ double wt[GJT][GJB + 1];
  __shared__ double bt[GJB][GJT];
  const int i0 = blockIdx.y * GJT, j0 = blockIdx.x * GJT;
  for (int e = threadIdx.x; e < GJT * GJB; e += blockDim.x) {
    const int r = e / GJB, m = e % GJB;
    wt[r][m] = i0 + r < nc ? W[(long long)(i0 + r) * GJB + m] : 0.0;
  }
  for (int e = threadIdx.x; e < GJB * GJT; e += blockDim.x) {
    const int m = e / GJT, c = e % GJT;
    bt[m][c] = (m < kb && j0 + c < nc) ? B[(long long)m * nc + j0 + c] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double acc[4][4] = {};
#pragma unroll 8
  for (int m = 0; m < GJB; ++m) {
    double a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = wt[ty + 16 * r][m];
#pragma unroll
    for (int c = 0; c < 4; ++c) b[c] = bt[m][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= nc) continue;
    const bool ik = i >= k0 && i < k0 + kb;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= nc) continue;
      double* xp = X + (long long)i * nc + j;
      if (j >= k0 && j < k0 + kb) *xp = -wt[ty + 16 * r][j - k0];
      else *xp = (ik ? 0.0 : *xp) - acc[r][c];
    }
  }
}

// the second nc x nc buffer also holds the pivot block, the panel and the
// copied pivot rows of the blocked inversion
size_t coarse_spare_doubles(int nc) {
  return std::max((size_t)nc * nc, (size_t)GJB * GJB + (size_t)2 * nc * GJB);
}

__global__ void k_coarse_to_f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// c = Phi^T r, one block per aggregate (fixed-order tree reduction)
constexpr int RESTRICT_THREADS = 512;

template <typename T, int DIM>
__global__ void __launch_bounds__(RESTRICT_THREADS) k_coarse_restrict(DevMesh m, int A, const T* __restrict__ rc,
                                                                      const T* __restrict__ r, T* __restrict__ cc,
                                                                      const int* skip) {
  // one thread per element node of the aggregate: its coordinates are read
  // once for its DIM unknowns; warp sums, then the warps' sums in order
  constexpr int NED = Shape<DIM>::ned, NEN = Shape<DIM>::nen, NM = n_modes<DIM>(), NT = RESTRICT_THREADS;
  constexpr int NW = NT / 32;
  __shared__ T red[NM][NW];
  if (skip && *skip) return;
  const int g = blockIdx.x, t = threadIdx.x;
  const long long q0 = (long long)g * A * NEN, q1 = (long long)min(m.ne, (g + 1) * A) * NEN;
  T s[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) s[k] = (T)0;
  for (long long q = q0 + t; q < q1; q += NT) {
    const int e = (int)(q / NEN), a = (int)(q - (long long)e * NEN);
    const unsigned dm = m.dirmask[e];
    const long long nb = (long long)e * NED + a * DIM;
    T X[DIM], v[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      X[k] = rc[nb + k];
      v[k] = ((dm >> (a * DIM + k)) & 1u) ? (T)0 : r[nb + k];
    }
#pragma unroll
    for (int comp = 0; comp < DIM; ++comp)
#pragma unroll
      for (int k = 0; k < NM; ++k) s[k] += rbm<DIM>(k, comp, X) * v[comp];
  }
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    T x = s[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) red[k][t >> 5] = x;
  }
  __syncthreads();
  if (t < NM) {
    T x = (T)0;
#pragma unroll
    for (int w = 0; w < NW; ++w) x += red[t][w];
    cc[g * NM + t] = x;
  }
}

// y = A0^-1 c, one warp per row
template <typename T>
__global__ void k_coarse_gemv(const T* __restrict__ Ainv, int nc, const T* __restrict__ cc, T* __restrict__ cy,
                              const int* skip) {
  if (skip && *skip) return;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= nc) return;
  const T* a = Ainv + (long long)row * nc;
  T s;
  using VT = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  if (nc % VN == 0) {
    // rows start on 16-byte boundaries: 16-byte loads, two independent sums
    const VT* a4 = reinterpret_cast<const VT*>(a);
    const VT* c4 = reinterpret_cast<const VT*>(cc);
    const int nv = nc / VN;
    VT s0 = Vec<T>::zero(), s1 = Vec<T>::zero();
    int j = lane;
    for (; j + 32 < nv; j += 64) {
      Vec<T>::madd(s0, a4[j], c4[j]);
      Vec<T>::madd(s1, a4[j + 32], c4[j + 32]);
    }
    for (; j < nv; j += 32) Vec<T>::madd(s0, a4[j], c4[j]);
    s = Vec<T>::hsum(s0) + Vec<T>::hsum(s1);
  } else {
    // four independent partial sums keep four loads in flight per lane
    T s0 = (T)0, s1 = (T)0, s2 = (T)0, s3 = (T)0;
    int j = lane;
    for (; j + 96 < nc; j += 128) {
      s0 += a[j] * cc[j];
      s1 += a[j + 32] * cc[j + 32];
      s2 += a[j + 64] * cc[j + 64];
      s3 += a[j + 96] * cc[j + 96];
    }
    for (; j < nc; j += 32) s0 += a[j] * cc[j];
    s = (s0 + s1) + (s2 + s3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) cy[row] = s;
}

// z += Phi y on the displacement unknowns
template <typename T, int DIM>
__global__ void k_coarse_prolong(DevMesh m, int A, const T* __restrict__ rc, const T* __restrict__ cy, T* z,
                                 const int* skip) {
  constexpr int NED = Shape<DIM>::ned, NM = n_modes<DIM>();
  // one thread per element node: its coordinates are read once for its DIM unknowns
  if (skip && *skip) return;
  constexpr int NEN = Shape<DIM>::nen;
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)m.ne * NEN) return;
  const int e = (int)(q / NEN), a = (int)(q % NEN);
  const unsigned dm = m.dirmask[e];
  const long long nb = (long long)e * NED + a * DIM;
  T X[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) X[k] = rc[nb + k];
  T y[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) y[k] = cy[(long long)(e / A) * NM + k];
#pragma unroll
  for (int comp = 0; comp < DIM; ++comp) {
    if ((dm >> (a * DIM + comp)) & 1u) continue;
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < NM; ++k) s += rbm<DIM>(k, comp, X) * y[k];
    z[nb + comp] += s;
  }
}

// ---------------------------------------------------------------- host side
void coarse_sizes(long long ne, int dim, int coarse_max, int* A, int* nagg, int* nc) {
  const int nm = dim == 2 ? 3 : 6;
  long long a = (ne * nm + coarse_max - 1) / std::max(coarse_max, 1);
  a = std::max<long long>(a, 8);
  *A = (int)a;
  *nagg = (int)((ne + a - 1) / a);
  *nc = *nagg * nm;
}

hf_status coarse_layout(hf_mesh* h) {
  int A, nagg, nc;
  coarse_sizes(h->ne, h->dim, h->opts.coarse_max, &A, &nagg, &nc);
  const bool same = h->rc64 && A == h->agg_size && nc == h->nc;
  h->coarse_dirty = true;
  if (same) return HF_OK;
  for (void* p : {(void*)h->agg_geo, (void*)h->rc64, (void*)h->rc32, (void*)h->A0a, (void*)h->A0b,
                  (void*)h->A0inv32, (void*)h->d_cthr, (void*)h->K64.cc, (void*)h->K64.cy, (void*)h->K32.cc,
                  (void*)h->K32.cy})
    dev_free(h, p);
  h->agg_size = A;
  h->nagg = nagg;
  h->nc = nc;
  const size_t nrc = (size_t)h->ne * h->ned, nc2 = (size_t)nc * nc;
  h->agg_geo = static_cast<double*>(dev_alloc(h, (size_t)nagg * 4 * sizeof(double)));
  h->rc64 = static_cast<double*>(dev_alloc(h, nrc * sizeof(double)));
  h->rc32 = static_cast<float*>(dev_alloc(h, nrc * sizeof(float)));
  h->A0a = static_cast<double*>(dev_alloc(h, nc2 * sizeof(double)));
  h->A0b = static_cast<double*>(dev_alloc(h, coarse_spare_doubles(nc) * sizeof(double)));
  h->A0inv32 = static_cast<float*>(dev_alloc(h, nc2 * sizeof(float)));
  h->d_cthr = static_cast<double*>(dev_alloc(h, sizeof(double)));
  h->K64.cc = static_cast<double*>(dev_alloc(h, (size_t)nc * sizeof(double)));
  h->K64.cy = static_cast<double*>(dev_alloc(h, (size_t)nc * sizeof(double)));
  h->K32.cc = static_cast<float*>(dev_alloc(h, (size_t)nc * sizeof(float)));
  h->K32.cy = static_cast<float*>(dev_alloc(h, (size_t)nc * sizeof(float)));
  if (!h->agg_geo || !h->rc64 || !h->rc32 || !h->A0a || !h->A0b || !h->A0inv32 || !h->d_cthr || !h->K64.cc ||
      !h->K64.cy || !h->K32.cc || !h->K32.cy)
    return set_error(h, HF_ERR_OOM, "coarse space");
  h->A0inv64 = nullptr;
  if (h->dim == 2) {
    note_launch();
    k_coarse_geo<2><<<nagg, 128, 0, h->stream>>>(h->d, A, h->agg_geo);
    note_launch();
    k_coarse_rc<2><<<(unsigned)((nrc + 255) / 256), 256, 0, h->stream>>>(h->d, A, h->agg_geo, h->rc64, h->rc32);
  } else {
    note_launch();
    k_coarse_geo<3><<<nagg, 128, 0, h->stream>>>(h->d, A, h->agg_geo);
    note_launch();
    k_coarse_rc<3><<<(unsigned)((nrc + 255) / 256), 256, 0, h->stream>>>(h->d, A, h->agg_geo, h->rc64, h->rc32);
  }
  return check_cuda(h, cudaGetLastError(), "coarse layout");
}

hf_status coarse_refactor(hf_mesh* h) {
  if (!h->coarse_dirty) return HF_OK;
  const int nc = h->nc, A = h->agg_size;
  const long long nc2 = (long long)nc * nc;
  prof_begin(h, PK_FACTOR);
  cudaMemsetAsync(h->A0a, 0, nc2 * sizeof(double), h->stream);
  if (h->dim == 2) {
    note_launch();
    k_coarse_build<2><<<h->nagg, 32, 0, h->stream>>>(h->d, A, nc, h->rc64, h->J64.dg, h->J64.off, h->A0a);
  } else {
    note_launch();
    k_coarse_build<3><<<h->nagg, 32, 0, h->stream>>>(h->d, A, nc, h->rc64, h->J64.dg, h->J64.off, h->A0a);
  }
  note_launch();
  k_coarse_thresh<<<1, 256, 0, h->stream>>>(h->A0a, nc, h->d_cthr);
  // blocked Gauss-Jordan in place on A0a; A0b holds the pivot block, the
  // panel W (nc x GJB) and the copied pivot rows B (GJB x nc)
  double* X = h->A0a;
  double* P = h->A0b;
  double* W = P + GJB * GJB;
  double* B = W + (size_t)nc * GJB;
  const dim3 tiles((unsigned)((nc + GJT - 1) / GJT), (unsigned)((nc + GJT - 1) / GJT));
  for (int k0 = 0; k0 < nc; k0 += GJB) {
    const int kb = std::min(GJB, nc - k0);
    note_launch();
    k_gj_pivot<<<1, GJB * GJB, 0, h->stream>>>(X, nc, k0, kb, h->d_cthr, P);
    note_launch();
    k_gj_panel<<<(unsigned)((nc + 7) / 8), 256, 0, h->stream>>>(X, nc, k0, kb, P, W, B);
    note_launch();
    k_gj_update<<<tiles, 256, 0, h->stream>>>(X, nc, k0, kb, W, B);
  }
  const unsigned blocks = (unsigned)((nc2 + 255) / 256);
  h->A0inv64 = X;
  note_launch();
  k_coarse_to_f<<<blocks, 256, 0, h->stream>>>(X, h->A0inv32, nc2);
  prof_end(h);
  h->coarse_dirty = false;
  return check_cuda(h, cudaGetLastError(), "coarse factor");
}

// A0 rebuilt into the buffer that does not hold the inverse (diagnostics)
hf_status coarse_rebuild_copy(hf_mesh* h, double* A0_host, double* inv_host, double* geo_host) {
  if (!h->opts.coarse || h->nc < 1) return set_error(h, HF_ERR_STATE, "no coarse level");
  hf_status s = coarse_refactor(h);
  if (s) return s;
  const int nc = h->nc;
  const long long nc2 = (long long)nc * nc;
  double* spare = h->A0inv64 == h->A0a ? h->A0b : h->A0a;
  cudaMemsetAsync(spare, 0, nc2 * sizeof(double), h->stream);
  note_launch();
  if (h->dim == 2)
    k_coarse_build<2><<<h->nagg, 32, 0, h->stream>>>(h->d, h->agg_size, nc, h->rc64, h->J64.dg, h->J64.off, spare);
  else
    k_coarse_build<3><<<h->nagg, 32, 0, h->stream>>>(h->d, h->agg_size, nc, h->rc64, h->J64.dg, h->J64.off, spare);
  if (A0_host) cudaMemcpyAsync(A0_host, spare, nc2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (inv_host) cudaMemcpyAsync(inv_host, h->A0inv64, nc2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (geo_host) cudaMemcpyAsync(geo_host, h->agg_geo, (size_t)h->nagg * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream);
  return check_cuda(h, cudaStreamSynchronize(h->stream), "coarse operator");
}

template <typename T> static const T* coarse_inverse(const hf_mesh* h);
template <> const double* coarse_inverse<double>(const hf_mesh* h) { return h->A0inv64; }
template <> const float* coarse_inverse<float>(const hf_mesh* h) { return h->A0inv32; }
template <typename T> static const T* coarse_coords(const hf_mesh* h);
template <> const double* coarse_coords<double>(const hf_mesh* h) { return h->rc64; }
template <> const float* coarse_coords<float>(const hf_mesh* h) { return h->rc32; }

template <typename T, int DIM>
void coarse_pre(hf_mesh* h, const Krylov<T>& K, const T* rin, const int* skip, cudaStream_t st) {
  note_launch();
  k_coarse_restrict<T, DIM><<<h->nagg, RESTRICT_THREADS, 0, st>>>(h->d, h->agg_size, coarse_coords<T>(h), rin,
                                                                    K.cc, skip);
  note_launch();
  k_coarse_gemv<T><<<(h->nc + 7) / 8, 256, 0, st>>>(coarse_inverse<T>(h), h->nc, K.cc, K.cy, skip);
}

template <typename T, int DIM> void coarse_post(hf_mesh* h, const Krylov<T>& K, T* z, const int* skip) {
  const long long n = h->ne * (long long)Shape<DIM>::nen;
  note_launch();
  k_coarse_prolong<T, DIM><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d, h->agg_size,
                                                                               coarse_coords<T>(h), K.cy, z, skip);
}

template void coarse_pre<float, 2>(hf_mesh*, const Krylov<float>&, const float*, const int*, cudaStream_t);
template void coarse_pre<float, 3>(hf_mesh*, const Krylov<float>&, const float*, const int*, cudaStream_t);
template void coarse_pre<double, 2>(hf_mesh*, const Krylov<double>&, const double*, const int*, cudaStream_t);
template void coarse_pre<double, 3>(hf_mesh*, const Krylov<double>&, const double*, const int*, cudaStream_t);
template void coarse_post<float, 2>(hf_mesh*, const Krylov<float>&, float*, const int*);
template void coarse_post<float, 3>(hf_mesh*, const Krylov<float>&, float*, const int*);
template void coarse_post<double, 2>(hf_mesh*, const Krylov<double>&, double*, const int*);
template void coarse_post<double, 3>(hf_mesh*, const Krylov<double>&, double*, const int*);

}  // namespace hfk
