// hf_assembly.cu - geometry, linear block build and nonlinear facet terms.
//
// Weak form (Eq. discreteElastoStatics): bulk int C eps(u):eps(v) plus, on
// intact interior facets, the IIPG consistency term <C eps(u)> n . [[v]] and
// the stability term (b/h) [[v]] (x) n : C : [[u]] (x) n, both switched off by
// alpha; cohesive traction alpha t(w).[[v]] (Eq. tsl) and fluid load
// -beta p n.[[v]].  Lubrication (Eq. discreteLubrication) on facets with
// beta = 1: int w^3/12mu grad p.grad q + (w - w^n)/dt q = Q0 q(x_in).
// The linear parts (bulk + intact facets) are assembled once into J_base and
// rebuilt only for elements whose facets change state; the nonlinear facet
// parts are reduced to small face-node matrices each Newton iteration.
#include "hf_internal.h"

namespace hfk {

// ---------------------------------------------------------------- geometry
template <int DIM>
__global__ void k_elem_geometry(DevMesh m) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  double X[DIM + 1][DIM];
  for (int i = 0; i < DIM + 1; ++i) {
    int g = m.enode[i * m.ne + e];
    for (int k = 0; k < DIM; ++k) X[i][k] = m.xyz[(long long)g * DIM + k];
  }
  // T = [X1-X0, ..., Xd-X0] (columns); grad lambda_i (i>=1) = rows of T^-1
  double T[DIM][DIM];
  for (int r = 0; r < DIM; ++r)
    for (int c = 0; c < DIM; ++c) T[r][c] = X[c + 1][r] - X[0][r];
  double inv[DIM][DIM], det;
  if (DIM == 2) {
    det = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    inv[0][0] = T[1][1] / det;
    inv[0][1] = -T[0][1] / det;
    inv[1][0] = -T[1][0] / det;
    inv[1][1] = T[0][0] / det;
  } else {
    double c00 = T[1][1] * T[2][2] - T[1][2] * T[2][1];
    double c01 = T[1][2] * T[2][0] - T[1][0] * T[2][2];
    double c02 = T[1][0] * T[2][1] - T[1][1] * T[2][0];
    det = T[0][0] * c00 + T[0][1] * c01 + T[0][2] * c02;
    // inverse = adj^T / det
    double a[3][3];
    a[0][0] = c00;
    a[1][0] = c01;
    a[2][0] = c02;
    a[0][1] = T[0][2] * T[2][1] - T[0][1] * T[2][2];
    a[1][1] = T[0][0] * T[2][2] - T[0][2] * T[2][0];
    a[2][1] = T[0][1] * T[2][0] - T[0][0] * T[2][1];
    a[0][2] = T[0][1] * T[1][2] - T[0][2] * T[1][1];
    a[1][2] = T[0][2] * T[1][0] - T[0][0] * T[1][2];
    a[2][2] = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) inv[r][c] = a[r][c] / det;
  }
  for (int k = 0; k < DIM; ++k) {
    double s = 0.0;
    for (int i = 0; i < DIM; ++i) {
      m.grad_lam[((i + 1) * DIM + k) * m.ne + e] = inv[i][k];
      s += inv[i][k];
    }
    m.grad_lam[(0 * DIM + k) * m.ne + e] = -s;
  }
  m.vol[e] = fabs(det) / (DIM == 2 ? 2.0 : 6.0);
}

template <int DIM>
__global__ void k_face_geometry(DevMesh m) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  int em = m.fe[f], ep = m.fe[m.nf + f];
  int i = m.fl[f];
  double g[DIM], gn = 0.0;
  for (int k = 0; k < DIM; ++k) {
    g[k] = m.grad_lam[(i * DIM + k) * m.ne + em];
    gn += g[k] * g[k];
  }
  gn = sqrt(gn);
  for (int k = 0; k < DIM; ++k) m.fnormal[k * m.nf + f] = -g[k] / gn;
  double area = DIM * m.vol[em] * gn;  // |f| = d |e| |grad lambda_i|
  m.farea[f] = area;
  double vmin = ep >= 0 ? fmin(m.vol[em], m.vol[ep]) : m.vol[em];
  m.fh[f] = vmin / area;
  // surface gradients of the face barycentrics from the facet vertices
  double V[DIM][DIM];
  for (int v = 0; v < DIM; ++v) {
    int gnode = m.enode[m.loc_m[v * m.nf + f] * m.ne + em];
    for (int k = 0; k < DIM; ++k) V[v][k] = m.xyz[(long long)gnode * DIM + k];
  }
  if (DIM == 2) {
    double t[2] = {V[1][0] - V[0][0], V[1][1] - V[0][1]};
    double tt = t[0] * t[0] + t[1] * t[1];
    for (int k = 0; k < 2; ++k) {
      m.fsg[(1 * DIM + k) * m.nf + f] = t[k] / tt;
      m.fsg[(0 * DIM + k) * m.nf + f] = -t[k] / tt;
    }
  } else {
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = V[1][k] - V[0][k];
      b[k] = V[2][k] - V[0][k];
    }
    double g11 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    double g12 = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    double g22 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double dd = g11 * g22 - g12 * g12;
    double i11 = g22 / dd, i12 = -g12 / dd, i22 = g11 / dd;
    for (int k = 0; k < 3; ++k) {
      double s1 = i11 * a[k] + i12 * b[k];
      double s2 = i12 * a[k] + i22 * b[k];
      m.fsg[(1 * DIM + k) * m.nf + f] = s1;
      m.fsg[(2 * DIM + k) * m.nf + f] = s2;
      m.fsg[(0 * DIM + k) * m.nf + f] = -(s1 + s2);
    }
  }
}

// ---------------------------------------------------------------- J_base rows
// One warp per listed element; lane r < ned owns matrix row r = a*DIM + k.
// Writes the dense block (bulk + intact-facet self terms) and, per facet slot,
// the compact neighbour block.  Dirichlet rows become identity rows.
template <int DIM>
__global__ void __launch_bounds__(128) k_build_rows(DevMesh m, Quad q, const int* elist, int nlist,
                                                    double* dg, double* off) {
  using S = Shape<DIM>;
  constexpr int NEN = S::nen, NED = S::ned, NFR = S::nfr, NFN = S::nfn;
  __shared__ double sh[4][4 * NEN * DIM + 2 * NEN];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int li = blockIdx.x * 4 + warp;
  if (li >= nlist) return;
  int e = elist[li];
  double* sG = sh[warp];                 // own gradients  [NEN*DIM]
  double* sGt = sG + NEN * DIM;          // neighbour gradients
  double* sN = sGt + NEN * DIM;          // own values
  double* sNt = sN + NEN;                // neighbour values
  const double lam = m.lam, mu = m.mu;
  const int r = lane, a = r / DIM, k = r % DIM;
  const bool active = r < NED;
  double acc[NED];
#pragma unroll
  for (int c = 0; c < NED; ++c) acc[c] = 0.0;
  double gl[(DIM + 1) * DIM];
  for (int t = 0; t < (DIM + 1) * DIM; ++t) gl[t] = m.grad_lam[t * m.ne + e];
  // bulk: sum_q |e| w_q [lam dNa_k dNb_l + mu (d_kl gNa.gNb + dNa_l dNb_k)]
  for (int qi = 0; qi < q.nq_v; ++qi) {
    __syncwarp();
    if (lane < NEN) {
      double G[NEN * DIM];
      p2_grads<DIM>(q.v_lam[qi], gl, G);
      for (int kk = 0; kk < DIM; ++kk) sG[lane * DIM + kk] = G[lane * DIM + kk];
    }
    __syncwarp();
    if (active) {
      double W = q.v_w[qi] * m.vol[e];
      double ga[DIM];
      for (int kk = 0; kk < DIM; ++kk) ga[kk] = sG[a * DIM + kk];
#pragma unroll
      for (int b = 0; b < NEN; ++b) {
        double gb[DIM], dot = 0.0;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) {
          gb[kk] = sG[b * DIM + kk];
          dot += ga[kk] * gb[kk];
        }
#pragma unroll
        for (int l = 0; l < DIM; ++l)
          acc[b * DIM + l] += W * (lam * ga[k] * gb[l] + mu * ((k == l ? dot : 0.0) + ga[l] * gb[k]));
      }
    }
  }
  unsigned dmask = m.dirmask[e];
  // facet slots
  for (int j = 0; j < DIM + 1; ++j) {
    int f = m.slot_face[j * m.ne + e];
    int nb = m.nbr[j * m.ne + e];
    int s = m.slot_side[j * m.ne + e];
    // face row index of this lane, or -1
    int rr = -1;
#pragma unroll
    for (int fa = 0; fa < NFN; ++fa)
      if (face_node<DIM>(j, fa) == a) rr = fa * DIM + k;
    double accn[NED];
#pragma unroll
    for (int c = 0; c < NED; ++c) accn[c] = 0.0;
    bool intact = (nb >= 0) && (m.alpha[f] == 0);
    if (intact) {
      double n[DIM];
      for (int kk = 0; kk < DIM; ++kk) n[kk] = m.fnormal[kk * m.nf + f];
      double pen = m.b_stab / m.fh[f];
      double sig_s = s == 0 ? -1.0 : 1.0;
      double glt[(DIM + 1) * DIM];
      for (int t = 0; t < (DIM + 1) * DIM; ++t) glt[t] = m.grad_lam[t * m.ne + nb];
      for (int qi = 0; qi < q.nq_l; ++qi) {
        __syncwarp();
        if (lane < NEN) {
          double lo[DIM + 1], lt[DIM + 1], N[NEN], G[NEN * DIM];
          face_to_elem_lam<DIM>(m, f, s, q.l_lam[qi], lo);
          face_to_elem_lam<DIM>(m, f, 1 - s, q.l_lam[qi], lt);
          p2_vals<DIM>(lo, N);
          p2_grads<DIM>(lo, gl, G);
          sN[lane] = N[lane];
          for (int kk = 0; kk < DIM; ++kk) sG[lane * DIM + kk] = G[lane * DIM + kk];
          p2_vals<DIM>(lt, N);
          p2_grads<DIM>(lt, glt, G);
          sNt[lane] = N[lane];
          for (int kk = 0; kk < DIM; ++kk) sGt[lane * DIM + kk] = G[lane * DIM + kk];
        }
        __syncwarp();
        if (active && rr >= 0) {
          double W = q.l_w[qi] * m.farea[f];
          double Na = sN[a];
#pragma unroll
          for (int b = 0; b < NEN; ++b) {
            double gs[DIM], gt[DIM], gsn = 0.0, gtn = 0.0;
#pragma unroll
            for (int kk = 0; kk < DIM; ++kk) {
              gs[kk] = sG[b * DIM + kk];
              gt[kk] = sGt[b * DIM + kk];
              gsn += gs[kk] * n[kk];
              gtn += gt[kk] * n[kk];
            }
            double Nbs = sN[b], Nbt = sNt[b];
#pragma unroll
            for (int l = 0; l < DIM; ++l) {
              double cc = (k == l ? mu : 0.0) + (lam + mu) * n[k] * n[l];
              double cons_s = lam * gs[l] * n[k] + mu * (n[l] * gs[k] + (k == l ? gsn : 0.0));
              double cons_t = lam * gt[l] * n[k] + mu * (n[l] * gt[k] + (k == l ? gtn : 0.0));
              acc[b * DIM + l] += W * Na * (0.5 * sig_s * cons_s + pen * Nbs * cc);
              accn[b * DIM + l] += W * Na * (0.5 * sig_s * cons_t - pen * Nbt * cc);
            }
          }
        }
      }
    }
    if (active && rr >= 0) {
      bool dir = (dmask >> r) & 1u;
      for (int c = 0; c < NED; ++c)
        off[((long long)(j * NED + c) * NFR + rr) * m.ne + e] = dir ? 0.0 : accn[c];
    }
  }
  if (active) {
    bool dir = (dmask >> r) & 1u;
    for (int c = 0; c < NED; ++c)
      dg[((long long)c * NED + r) * m.ne + e] = dir ? (c == r ? 1.0 : 0.0) : acc[c];
  }
}

// Neumann load f_ext = sum over traction facets of int tbar . N_a
template <int DIM>
__global__ void k_neumann(DevMesh m, Quad q, const double* ftrac, const signed char* fneu) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  for (int j = 0; j < DIM + 1; ++j) {
    int f = m.slot_face[j * m.ne + e];
    if (f < 0 || !fneu[f]) continue;
    for (int qi = 0; qi < q.nq_l; ++qi) {
      double lo[DIM + 1], N[Shape<DIM>::nen];
      face_to_elem_lam<DIM>(m, f, 0, q.l_lam[qi], lo);
      p2_vals<DIM>(lo, N);
      double W = q.l_w[qi] * m.farea[f];
      for (int a = 0; a < Shape<DIM>::nen; ++a)
        for (int k = 0; k < DIM; ++k)
          m.fext[(long long)e * Shape<DIM>::ned + a * DIM + k] += W * N[a] * ftrac[k * m.nf + f];
    }
  }
}

// ---------------------------------------------------------------- nonlinear facets
// One warp per facet with alpha or beta set.  All lanes evaluate the facet
// kinematics at each quadrature point; lane l accumulates matrix entries
// l, l+32 of the face-node matrices and lanes < nfn the vectors.
template <int DIM>
__global__ void __launch_bounds__(128) k_face_nl(DevMesh m, Quad q, const double* __restrict__ X) {
  using S = Shape<DIM>;
  using L = NL<DIM>;
  constexpr int F = S::nfn, NED = S::ned;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int li = blockIdx.x * 4 + warp;
  if (li >= m.n_nl) return;
  int f = m.nl_faces[li];
  int em = m.fe[f], ep = m.fe[m.nf + f], j = m.fl[f];
  bool al = m.alpha[f] != 0, be = m.beta[f] != 0;
  double n[DIM];
  for (int k = 0; k < DIM; ++k) n[k] = m.fnormal[k * m.nf + f];
  double sg[DIM * DIM];
  for (int t = 0; t < DIM * DIM; ++t) sg[t] = m.fsg[t * m.nf + f];
  double wn[F], P[F], wo[F];
  for (int a = 0; a < F; ++a) {
    int lm = m.loc_m[a * m.nf + f], lp = m.loc_p[a * m.nf + f];
    double s = 0.0;
    for (int k = 0; k < DIM; ++k)
      s += (X[(long long)ep * NED + lp * DIM + k] - X[(long long)em * NED + lm * DIM + k]) * n[k];
    wn[a] = s;
    int pd = m.fpdof[a * m.nf + f];
    P[a] = pd >= 0 ? X[m.nu + pd] : 0.0;
    wo[a] = m.w_old[a * m.nf + f];
  }
  double kp = m.b_stab / m.fh[f] * (m.lam + 2.0 * m.mu);
  double area = m.farea[f];
  double mu12 = 12.0 * m.mu_f;
  // accumulators: entries pi = lane, lane + 32 of the F*F matrices
  double aT[2] = {0, 0}, aM[2] = {0, 0}, aC[2] = {0, 0}, aD[2] = {0, 0};
  double vc = 0.0, vp = 0.0, vf = 0.0;
  for (int qi = 0; qi < q.nq_f; ++qi) {
    double phi[F], G[F * DIM];
    face_vals<DIM>(j, q.f_lam[qi], phi);
    face_grads<DIM>(j, q.f_lam[qi], sg, G);
    double w = 0.0, p = 0.0, wold = 0.0, gp[DIM] = {};
    for (int a = 0; a < F; ++a) {
      w += phi[a] * wn[a];
      p += phi[a] * P[a];
      wold += phi[a] * wo[a];
      for (int k = 0; k < DIM; ++k) gp[k] += G[a * DIM + k] * P[a];
    }
    double W = q.f_w[qi] * area;
    double T = 0.0, dT = 0.0;
    if (al) tsl(w, m.sigma_c, m.delta_c, kp, T, dT);
    double wp = w > 0.0 ? w : 0.0;
    double k3 = wp * wp * wp / mu12, dk3 = 3.0 * wp * wp / mu12;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int pi = lane + 32 * h;
      if (pi < F * F) {
        int ra = pi / F, cb = pi % F;
        double gpa = 0.0, gg = 0.0;
        for (int k = 0; k < DIM; ++k) {
          gpa += gp[k] * G[ra * DIM + k];
          gg += G[ra * DIM + k] * G[cb * DIM + k];
        }
        aT[h] += W * dT * phi[ra] * phi[cb];
        aM[h] += W * phi[ra] * phi[cb];
        aC[h] += W * (dk3 * gpa + phi[ra] / m.dt) * phi[cb];
        aD[h] += W * k3 * gg;
      }
    }
    if (lane < F) {
      double gpa = 0.0;
      for (int k = 0; k < DIM; ++k) gpa += gp[k] * G[lane * DIM + k];
      vc += W * T * phi[lane];
      vp += W * p * phi[lane];
      vf += W * (k3 * gpa + (w - wold) / m.dt * phi[lane]);
    }
  }
  double* rec = m.nl + (long long)f * S::nld;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int pi = lane + 32 * h;
    if (pi < F * F) {
      rec[L::Tm + pi] = al ? aT[h] : 0.0;
      rec[L::Mm + pi] = be ? aM[h] : 0.0;
      rec[L::Cs + pi] = be ? aC[h] : 0.0;
      rec[L::Dm + pi] = be ? aD[h] : 0.0;
    }
  }
  if (lane < F) {
    rec[L::rc + lane] = al ? vc : 0.0;
    rec[L::rp + lane] = be ? vp : 0.0;
    rec[L::rf + lane] = be ? vf : 0.0;
  }
}

// ---------------------------------------------------------------- criterion
// Normal DG traction n.<sigma(u)>n + (b/h)(lambda + 2mu) w at each facet
// quadrature point of crackable intact facets; alpha := 1 above sigma_c.
template <int DIM>
__global__ void k_criterion(DevMesh m, Quad q, const double* __restrict__ X, double* tmax_out,
                            int* n_new) {
  using S = Shape<DIM>;
  constexpr int NEN = S::nen, NED = S::ned, F = S::nfn;
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  if (!m.crack[f] || m.alpha[f]) {
    if (tmax_out) tmax_out[f] = -INFINITY;
    return;
  }
  int el[2] = {m.fe[f], m.fe[m.nf + f]};
  double n[DIM];
  for (int k = 0; k < DIM; ++k) n[k] = m.fnormal[k * m.nf + f];
  double wn[F];
  for (int a = 0; a < F; ++a) {
    int lm = m.loc_m[a * m.nf + f], lp = m.loc_p[a * m.nf + f];
    double s = 0.0;
    for (int k = 0; k < DIM; ++k)
      s += (X[(long long)el[1] * NED + lp * DIM + k] - X[(long long)el[0] * NED + lm * DIM + k]) * n[k];
    wn[a] = s;
  }
  int j = m.fl[f];
  double pen = m.b_stab / m.fh[f] * (m.lam + 2.0 * m.mu);
  double best = -INFINITY;
  for (int qi = 0; qi < q.nq_f; ++qi) {
    double phi[F];
    face_vals<DIM>(j, q.f_lam[qi], phi);
    double w = 0.0;
    for (int a = 0; a < F; ++a) w += phi[a] * wn[a];
    double tn = 0.0;
    for (int s = 0; s < 2; ++s) {
      int e = el[s];
      double lam_e[DIM + 1], gl[(DIM + 1) * DIM], G[NEN * DIM];
      face_to_elem_lam<DIM>(m, f, s, q.f_lam[qi], lam_e);
      for (int t = 0; t < (DIM + 1) * DIM; ++t) gl[t] = m.grad_lam[t * m.ne + e];
      p2_grads<DIM>(lam_e, gl, G);
      double gu[DIM][DIM] = {};  // gu[k][i] = d u_k / d x_i
      for (int a = 0; a < NEN; ++a)
        for (int k = 0; k < DIM; ++k) {
          double ua = X[(long long)e * NED + a * DIM + k];
          for (int i = 0; i < DIM; ++i) gu[k][i] += ua * G[a * DIM + i];
        }
      double tr = 0.0;
      for (int k = 0; k < DIM; ++k) tr += gu[k][k];
      // n . sigma n with sigma = lam tr(eps) I + mu (grad u + grad u^T)
      double sn = m.lam * tr;
      for (int k = 0; k < DIM; ++k)
        for (int i = 0; i < DIM; ++i) sn += m.mu * (gu[k][i] + gu[i][k]) * n[k] * n[i];
      tn += 0.5 * sn;
    }
    tn += pen * w;
    best = fmax(best, tn);
  }
  if (tmax_out) tmax_out[f] = best;
  if (n_new && best > m.sigma_c) {
    m.alpha[f] = 1;
    atomicAdd(n_new, 1);
  }
}

// ---------------------------------------------------------------- openings / end of step
template <int DIM>
__global__ void k_face_openings(DevMesh m, const double* __restrict__ X, double* wout) {
  using S = Shape<DIM>;
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  int em = m.fe[f], ep = m.fe[m.nf + f];
  for (int a = 0; a < S::nfn; ++a) {
    double s = 0.0;
    if (ep >= 0) {
      int lm = m.loc_m[a * m.nf + f], lp = m.loc_p[a * m.nf + f];
      for (int k = 0; k < DIM; ++k)
        s += (X[(long long)ep * S::ned + lp * DIM + k] - X[(long long)em * S::ned + lm * DIM + k]) *
             m.fnormal[k * m.nf + f];
    }
    wout[a * m.nf + f] = s;
  }
}

// beta := 1 where alpha = 1 and the opening exceeds delta_f at a facet
// quadrature point; then w^n := w^{n+1} at the face nodes
template <int DIM>
__global__ void k_accept(DevMesh m, Quad q, const double* __restrict__ X, int* n_new) {
  using S = Shape<DIM>;
  constexpr int F = S::nfn;
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  int em = m.fe[f], ep = m.fe[m.nf + f];
  double wn[F];
  for (int a = 0; a < F; ++a) {
    double s = 0.0;
    if (ep >= 0) {
      int lm = m.loc_m[a * m.nf + f], lp = m.loc_p[a * m.nf + f];
      for (int k = 0; k < DIM; ++k)
        s += (X[(long long)ep * S::ned + lp * DIM + k] - X[(long long)em * S::ned + lm * DIM + k]) *
             m.fnormal[k * m.nf + f];
    }
    wn[a] = s;
  }
  if (m.crack[f] && m.alpha[f] && !m.beta[f]) {
    double best = -INFINITY;
    for (int qi = 0; qi < q.nq_f; ++qi) {
      double phi[F];
      face_vals<DIM>(m.fl[f], q.f_lam[qi], phi);
      double w = 0.0;
      for (int a = 0; a < F; ++a) w += phi[a] * wn[a];
      best = fmax(best, w);
    }
    if (best > m.delta_f) {
      m.beta[f] = 1;
      atomicAdd(n_new, 1);
    }
  }
  for (int a = 0; a < F; ++a) m.w_old[a * m.nf + f] = wn[a];
}

// c^n = 12 mu (L / max w^n)^3 over the face nodes of crackable facets
__global__ void k_fluid_scale(DevMesh m, int enabled, double L_ref) {
  __shared__ double sm[1024];
  double mx = 0.0;
  for (long long i = threadIdx.x; i < (long long)m.nf * m.nfn; i += blockDim.x) {
    int f = (int)(i % m.nf);
    if (m.crack[f]) mx = fmax(mx, m.w_old[i]);
  }
  sm[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double w = sm[0];
    double c = 1.0;
    if (enabled && w > 0.0) {
      double r = w / L_ref;
      c = 12.0 * m.mu_f / (r * r * r);
    }
    m.scal[0] = c;
  }
}

// ---------------------------------------------------------------- launchers
template <int DIM>
void launch_geometry(const DevMesh& m, cudaStream_t st) {
  { note_launch(); k_elem_geometry<DIM><<<(m.ne + 127) / 128, 128, 0, st>>>(m); }
  { note_launch(); k_face_geometry<DIM><<<(m.nf + 127) / 128, 128, 0, st>>>(m); }
}
template <int DIM>
void launch_build_rows(const DevMesh& m, const Quad& q, const int* elist, int n, double* dg, double* off,
                       cudaStream_t st) {
  if (n > 0) { note_launch(); k_build_rows<DIM><<<(n + 3) / 4, 128, 0, st>>>(m, q, elist, n, dg, off); }
}
template <int DIM>
void launch_neumann(const DevMesh& m, const Quad& q, const double* ftrac, const signed char* fneu,
                    cudaStream_t st) {
  { note_launch(); k_neumann<DIM><<<(m.ne + 127) / 128, 128, 0, st>>>(m, q, ftrac, fneu); }
}
template <int DIM>
void launch_face_nl(const DevMesh& m, const Quad& q, const double* X, cudaStream_t st) {
  if (m.n_nl > 0) { note_launch(); k_face_nl<DIM><<<(m.n_nl + 3) / 4, 128, 0, st>>>(m, q, X); }
}
template <int DIM>
void launch_criterion(const DevMesh& m, const Quad& q, const double* X, double* tmax, int* n_new,
                      cudaStream_t st) {
  { note_launch(); k_criterion<DIM><<<(m.nf + 127) / 128, 128, 0, st>>>(m, q, X, tmax, n_new); }
}
template <int DIM>
void launch_openings(const DevMesh& m, const double* X, double* w, cudaStream_t st) {
  { note_launch(); k_face_openings<DIM><<<(m.nf + 127) / 128, 128, 0, st>>>(m, X, w); }
}
template <int DIM>
void launch_accept(const DevMesh& m, const Quad& q, const double* X, int* n_new, cudaStream_t st) {
  { note_launch(); k_accept<DIM><<<(m.nf + 127) / 128, 128, 0, st>>>(m, q, X, n_new); }
}
void launch_fluid_scale(const DevMesh& m, int enabled, double L_ref, cudaStream_t st) {
  { note_launch(); k_fluid_scale<<<1, 1024, 0, st>>>(m, enabled, L_ref); }
}

#define HF_INST(DIM)                                                                             \
  template void launch_geometry<DIM>(const DevMesh&, cudaStream_t);                              \
  template void launch_build_rows<DIM>(const DevMesh&, const Quad&, const int*, int, double*,    \
                                       double*, cudaStream_t);                                   \
  template void launch_neumann<DIM>(const DevMesh&, const Quad&, const double*,                  \
                                    const signed char*, cudaStream_t);                           \
  template void launch_face_nl<DIM>(const DevMesh&, const Quad&, const double*, cudaStream_t);   \
  template void launch_criterion<DIM>(const DevMesh&, const Quad&, const double*, double*, int*, \
                                      cudaStream_t);                                             \
  template void launch_openings<DIM>(const DevMesh&, const double*, double*, cudaStream_t);      \
  template void launch_accept<DIM>(const DevMesh&, const Quad&, const double*, int*, cudaStream_t);
HF_INST(2)
HF_INST(3)

}  // namespace hfk
