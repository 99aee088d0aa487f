// hf_api.cu - the C ABI of include/hf.h: mesh set-up, state transfer and the
// Newton-step orchestration.  Host code here only moves data, builds index
// structures (element order, facet slots, pressure numbering, subdomain level
// schedule, quadrature nodes) and sequences kernels; every term of the
// residual, the Jacobian and the solve is computed on the GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "hf_internal.h"

using namespace hfk;

namespace hfk {
long long& launch_counter() {
  thread_local long long n = 0;
  return n;
}
static std::atomic<long long> g_launches{0};
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long total_launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hfk

namespace hfk {
void launch_neg(hf_mesh* h, const double* a, double* b);
void launch_precond64(hf_mesh* h, const double* r, double* z);
}

// ---------------------------------------------------------------- quadrature
// Gauss rules on [0,1] for the weight (1-t)^a: nodes are the roots of the
// degree-n Jacobi polynomial P_n^(a,0) (three-term recurrence, bracketed by
// sign changes and bisected), weights solve the moment equations
// sum_i w_i t_i^k = int_0^1 (1-t)^a t^k dt = k! a! / (k+a+1)!.
static double jacobi_p(int n, double a, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * (a + (a + 2.0) * x);
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a;
    double a1 = 2.0 * k * (k + a) * (c - 2.0);
    double a2 = (c - 1.0) * a * a;
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (k + a - 1.0) * (k - 1.0) * c;
    double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static void gauss01(int n, int a, double* t, double* w) {
  std::vector<double> roots;
  const int M = 20000;
  double xprev = -1.0, fprev = jacobi_p(n, a, -1.0 + 1e-15);
  for (int i = 1; i <= M; ++i) {
    double x = -1.0 + 2.0 * i / M;
    if (i == M) x = 1.0 - 1e-15;
    double fx = jacobi_p(n, a, x);
    if ((fprev < 0) != (fx < 0)) {
      double lo = xprev, hi = x, flo = fprev;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = jacobi_p(n, a, mid);
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      roots.push_back(0.5 * (lo + hi));
    }
    xprev = x;
    fprev = fx;
  }
  for (int i = 0; i < n; ++i) t[i] = 0.5 * (roots[i] + 1.0);
  // moments and a Vandermonde solve in long double
  long double A[8][9];
  for (int k = 0; k < n; ++k) {
    long double mom = 1.0L;  // k! a! / (k+a+1)!
    long double num = 1.0L, den = 1.0L;
    for (int q = 2; q <= k; ++q) num *= q;
    for (int q = 2; q <= a; ++q) num *= q;
    for (int q = 2; q <= k + a + 1; ++q) den *= q;
    mom = num / den;
    for (int i = 0; i < n; ++i) A[k][i] = powl((long double)t[i], k);
    A[k][n] = mom;
  }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r][c]) > fabsl(A[p][c])) p = r;
    for (int q = 0; q <= n; ++q) std::swap(A[c][q], A[p][q]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      long double f = A[r][c] / A[c][c];
      for (int q = c; q <= n; ++q) A[r][q] -= f * A[c][q];
    }
  }
  for (int i = 0; i < n; ++i) w[i] = (double)(A[i][n] / A[i][i]);
}

// rule on the reference s-simplex: barycentric coordinates, weights summing
// to 1; s = 1 Gauss-Legendre, s = 2, 3 collapsed-coordinate products
static int simplex_rule(int s, int n, double (*lam)[4], double* wts) {
  double u[8], wu[8], v[8], wv[8], t[8], wt[8];
  int nq = 0;
  if (s == 1) {
    gauss01(n, 0, t, wt);
    for (int i = 0; i < n; ++i) {
      lam[nq][0] = 1.0 - t[i];
      lam[nq][1] = t[i];
      wts[nq++] = wt[i];
    }
  } else if (s == 2) {
    gauss01(n, 1, u, wu);
    gauss01(n, 0, v, wv);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double x1 = u[i], x2 = v[j] * (1.0 - u[i]);
        lam[nq][0] = 1.0 - x1 - x2;
        lam[nq][1] = x1;
        lam[nq][2] = x2;
        wts[nq++] = wu[i] * wv[j];
      }
  } else {
    gauss01(n, 2, u, wu);
    gauss01(n, 1, v, wv);
    gauss01(n, 0, t, wt);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          double x1 = u[i], x2 = v[j] * (1.0 - u[i]), x3 = t[k] * (1.0 - u[i]) * (1.0 - v[j]);
          lam[nq][0] = 1.0 - x1 - x2 - x3;
          lam[nq][1] = x1;
          lam[nq][2] = x2;
          lam[nq][3] = x3;
          wts[nq++] = wu[i] * wv[j] * wt[k];
        }
  }
  double sum = 0.0;
  for (int i = 0; i < nq; ++i) sum += wts[i];
  for (int i = 0; i < nq; ++i) wts[i] /= sum;
  return nq;
}

static void build_quad(int dim, Quad& q) {
  double lam[128][4], w[128];
  // nonlinear facet rule: 5 points per direction (matches the facet convention of hf.h)
  q.nq_f = simplex_rule(dim - 1, 5, lam, w);
  for (int i = 0; i < q.nq_f; ++i) {
    for (int k = 0; k < 3; ++k) q.f_lam[i][k] = lam[i][k];
    q.f_w[i] = w[i];
  }
  // linear facet terms are polynomials of degree <= 4: 3 points per direction
  q.nq_l = simplex_rule(dim - 1, 3, lam, w);
  for (int i = 0; i < q.nq_l; ++i) {
    for (int k = 0; k < 3; ++k) q.l_lam[i][k] = lam[i][k];
    q.l_w[i] = w[i];
  }
  // bulk stiffness of affine P2 elements has degree 2: 2 points per direction
  q.nq_v = simplex_rule(dim, 2, lam, w);
  for (int i = 0; i < q.nq_v; ++i) {
    for (int k = 0; k < 4; ++k) q.v_lam[i][k] = lam[i][k];
    q.v_w[i] = w[i];
  }
}

// ---------------------------------------------------------------- helpers
namespace hfk {
void* dev_alloc(hf_mesh* h, size_t bytes) {
  bytes = (std::max<size_t>(bytes, 1) + 255) / 256 * 256;
  void* raw = nullptr;
  if (cudaMallocAsync(&raw, bytes + 256, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  void* base = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(raw) + 255) & ~uintptr_t(255));
  h->allocs.push_back({raw, base, bytes});
  h->bytes_allocated += (long long)bytes;
  return base;
}

void dev_free(hf_mesh* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i].base == p) {
      cudaFreeAsync(h->allocs[i].raw, h->stream);
      h->bytes_allocated -= (long long)h->allocs[i].bytes;
      h->allocs[i] = h->allocs.back();
      h->allocs.pop_back();
      return;
    }
}
}  // namespace hfk

template <typename T> static T* upload(hf_mesh* h, const std::vector<T>& v) {
  void* p = dev_alloc(h, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (!p) return nullptr;
  if (!v.empty()) cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream);
  return reinterpret_cast<T*>(p);
}
template <typename T> static T* dzeros(hf_mesh* h, size_t n) {
  n = std::max<size_t>(n, 1);
  void* p = dev_alloc(h, n * sizeof(T));
  if (!p) return nullptr;
  cudaMemsetAsync(p, 0, n * sizeof(T), h->stream);
  return reinterpret_cast<T*>(p);
}

static uint64_t spread2(uint64_t x) {
  x &= 0xffffffffULL;
  x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x << 2)) & 0x3333333333333333ULL;
  x = (x | (x << 1)) & 0x5555555555555555ULL;
  return x;
}
static uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}

static int fnode(int dim, int j, int a) { return dim == 2 ? fn2(j, a) : fn3(j, a); }

#define HF_GUARD(h)                                                                  \
  do {                                                                               \
    if (!(h)) return HF_ERR_INVALID_ARG;                                             \
    if ((h)->poisoned) return set_error((h), HF_ERR_STATE, "handle poisoned: " + (h)->err); \
  } while (0)

#define HF_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return check_cuda((h), e_, #call); \
  } while (0)

// ---------------------------------------------------------------- lists
// Rebuild the facet-state dependent index data from the host copies of alpha
// and beta: nonlinear facet list, element slot masks, active pressures and the
// subdomains whose factor changes every Newton iteration.
static hf_status rebuild_lists(hf_mesh* h) {
  int ne = (int)h->ne, nf = (int)h->nf, np = (int)h->np, nsl = h->dim + 1;
  std::vector<int> nl;
  for (int f = 0; f < nf; ++f)
    if (h->h_crack[f] && (h->h_alpha[f] || h->h_beta[f])) nl.push_back(f);
  std::vector<unsigned char> nlmask(ne, 0);
  std::vector<char> sd_coh(h->d.nsd, 0);
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < nsl; ++j) {
      int f = h->h_slot_face[j * ne + e];
      if (f < 0 || h->h_nbr[j * ne + e] < 0 || !h->h_crack[f]) continue;
      if (h->h_alpha[f]) {
        nlmask[e] |= 1u << j;
        sd_coh[h->sd_of[e]] = 1;
      }
      if (h->h_beta[f]) nlmask[e] |= 1u << (4 + j);
    }
  std::vector<signed char> pact(np, 0);
  for (int f = 0; f < nf; ++f) {
    if (!h->h_crack[f] || !h->h_beta[f]) continue;
    for (int a = 0; a < h->nfn; ++a) {
      int pd = h->hp_fpdof[a * nf + f];
      if (pd >= 0) pact[pd] = 1;
    }
  }
  h->sd_always.clear();
  for (int s = 0; s < h->d.nsd; ++s)
    if (sd_coh[s]) h->sd_always.push_back(s);
  if (h->nl_cap < (int)nl.size() || !h->d.nl_faces) {
    h->nl_cap = std::max<int>((int)nl.size(), 64);
    dev_free(h, h->d.nl_faces);
    h->d.nl_faces = dzeros<int>(h, h->nl_cap);
    if (!h->d.nl_faces) return set_error(h, HF_ERR_OOM, "nonlinear facet list");
  }
  h->d.n_nl = (int)nl.size();
  if (!nl.empty()) cudaMemcpyAsync(h->d.nl_faces, nl.data(), nl.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->d.nlmask, nlmask.data(), ne, cudaMemcpyHostToDevice, h->stream);
  if (np > 0) cudaMemcpyAsync(h->d.p_active, pact.data(), np, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->d.alpha, h->h_alpha.data(), nf, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->d.beta, h->h_beta.data(), nf, cudaMemcpyHostToDevice, h->stream);
  return check_cuda(h, cudaGetLastError(), "rebuild_lists");
}

// subdomains of G consecutive elements and their level schedule
static hf_status build_subdomains(hf_mesh* h, int G) {
  int ne = (int)h->ne, nsl = h->dim + 1;
  G = std::max(1, std::min(G, 256));
  int nsd = (ne + G - 1) / G;
  std::vector<int> level(ne, 0), sd_elems(ne), sd_lvl, sd_base(nsd), sd_nlvl(nsd);
  std::vector<unsigned char> low(ne, 0), up(ne, 0);
  h->sd_of.assign(ne, 0);
  for (int s = 0; s < nsd; ++s) {
    int b = s * G, c = std::min(G, ne - b);
    int maxl = 0;
    for (int e = b; e < b + c; ++e) {
      h->sd_of[e] = s;
      int l = 0;
      for (int j = 0; j < nsl; ++j) {
        int nb = h->h_nbr[j * ne + e];
        if (nb >= b && nb < e) {
          l = std::max(l, level[nb] + 1);
          low[e] |= 1u << j;
        } else if (nb > e && nb < b + c) {
          up[e] |= 1u << j;
        }
      }
      level[e] = l;
      maxl = std::max(maxl, l);
    }
    std::vector<int> idx(c);
    std::iota(idx.begin(), idx.end(), b);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return level[x] < level[y]; });
    for (int i = 0; i < c; ++i) sd_elems[b + i] = idx[i];
    sd_base[s] = (int)sd_lvl.size();
    sd_nlvl[s] = maxl + 1;
    int pos = b;
    for (int l = 0; l <= maxl; ++l) {
      sd_lvl.push_back(pos);
      while (pos < b + c && level[sd_elems[pos]] == l) ++pos;
    }
    sd_lvl.push_back(b + c);
  }
  h->G = G;
  h->d.G = G;
  h->d.nsd = nsd;
  for (void* old : {(void*)h->d.sd_elems, (void*)h->d.sd_lvl, (void*)h->d.sd_lvl_base, (void*)h->d.sd_nlvl})
    dev_free(h, old);
  h->d.sd_elems = upload(h, sd_elems);
  h->d.sd_lvl = upload(h, sd_lvl);
  h->d.sd_lvl_base = upload(h, sd_base);
  h->d.sd_nlvl = upload(h, sd_nlvl);
  if (!h->d.lowmask) h->d.lowmask = dzeros<unsigned char>(h, ne);
  if (!h->d.upmask) h->d.upmask = dzeros<unsigned char>(h, ne);
  if (!h->d_sdlist) h->d_sdlist = dzeros<int>(h, ne);
  if (!h->d.sd_elems || !h->d.sd_lvl || !h->d.sd_lvl_base || !h->d.sd_nlvl || !h->d.lowmask || !h->d.upmask ||
      !h->d_sdlist)
    return set_error(h, HF_ERR_OOM, "subdomain structures");
  cudaMemcpyAsync(h->d.lowmask, low.data(), ne, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->d.upmask, up.data(), ne, cudaMemcpyHostToDevice, h->stream);
  h->levels_max = 0;
  for (int s = 0; s < nsd; ++s) h->levels_max = std::max(h->levels_max, sd_nlvl[s]);
  h->n_subdomain_slots = 0;
  h->n_interior_slots = 0;
  std::vector<long long> rec_fwd(ne), rec_bwd(ne);
  const long long bs = (long long)h->ned * h->nfr, dsz = (long long)h->ned * h->ned;
  long long off = 0;
  for (int e = 0; e < ne; ++e) {
    h->n_subdomain_slots += __builtin_popcount((unsigned)(low[e] | up[e]));
    for (int j = 0; j < nsl; ++j) h->n_interior_slots += h->h_nbr[j * ne + e] >= 0;
  }
  for (int s = 0; s < nsd; ++s) {
    int b = s * G, c = std::min(G, ne - b);
    for (int k = 0; k < c; ++k) {  // forward stream, level order
      int e = sd_elems[b + k];
      rec_fwd[e] = off;
      off += __builtin_popcount((unsigned)low[e]) * bs;
    }
    for (int k = c - 1; k >= 0; --k) {  // backward stream, reverse level order
      int e = sd_elems[b + k];
      rec_bwd[e] = off;
      off += __builtin_popcount((unsigned)up[e]) * bs + dsz;
    }
  }
  // per position in level order: local element id, lower/upper slot masks and
  // the local ids of the four slot neighbours (255 outside the subdomain)
  std::vector<unsigned char> task((size_t)ne * 8, 255);
  std::vector<long long> sd_fwd(nsd), sd_bwd(nsd);
  for (int s = 0; s < nsd; ++s) {
    int b = s * G, c = std::min(G, ne - b);
    for (int k = 0; k < c; ++k) {
      int e = sd_elems[b + k];
      unsigned char* t = &task[(size_t)(b + k) * 8];
      t[0] = (unsigned char)(e - b);
      t[1] = low[e];
      t[2] = up[e];
      for (int j = 0; j < nsl; ++j) {
        int nb = h->h_nbr[j * ne + e];
        t[4 + j] = (nb >= b && nb < b + c) ? (unsigned char)(nb - b) : 255;
      }
    }
    sd_fwd[s] = c ? rec_fwd[sd_elems[b]] : 0;
    sd_bwd[s] = c ? rec_bwd[sd_elems[b + c - 1]] : 0;
  }
  for (void* old : {(void*)h->d.rec_fwd, (void*)h->d.rec_bwd, (void*)h->d.sd_task, (void*)h->d.sd_fwd,
                    (void*)h->d.sd_bwd})
    dev_free(h, old);
  h->d.rec_fwd = upload(h, rec_fwd);
  h->d.rec_bwd = upload(h, rec_bwd);
  h->d.sd_task = upload(h, task);
  h->d.sd_fwd = upload(h, sd_fwd);
  h->d.sd_bwd = upload(h, sd_bwd);
  if (!h->d.rec_fwd || !h->d.rec_bwd || !h->d.sd_task || !h->d.sd_fwd || !h->d.sd_bwd)
    return set_error(h, HF_ERR_OOM, "ILU record offsets");
  return check_cuda(h, cudaGetLastError(), "build_subdomains");
}

static void invalidate_graphs(hf_mesh* h) {
  if (h->graph64) cudaGraphExecDestroy(h->graph64);
  if (h->graph32) cudaGraphExecDestroy(h->graph32);
  h->graph64 = h->graph32 = nullptr;
  for (auto* v : {&h->gev64, &h->gev32}) {
    for (GraphEv& g : *v) {
      cudaEventDestroy(g.a);
      cudaEventDestroy(g.b);
    }
    v->clear();
  }
}

static std::vector<int> all_subdomains(hf_mesh* h) {
  std::vector<int> v(h->d.nsd);
  std::iota(v.begin(), v.end(), 0);
  return v;
}

// rebuild J_base rows of the given elements and mark their subdomains dirty
static hf_status rebuild_rows(hf_mesh* h, const std::vector<int>& elems) {
  if (elems.empty()) return HF_OK;
  cudaMemcpyAsync(h->d_elist, elems.data(), elems.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (h->dim == 2) launch_build_rows<2>(h->d, h->q, h->d_elist, (int)elems.size(), h->J64.dg, h->J64.off, h->stream);
  else launch_build_rows<3>(h->d, h->q, h->d_elist, (int)elems.size(), h->J64.dg, h->J64.off, h->stream);
  h->j32_valid = false;
  h->coarse_dirty = true;
  for (int e : elems) h->sd_dirty.push_back(h->sd_of[e]);
  return check_cuda(h, cudaGetLastError(), "build_rows");
}

static hf_status refactor(hf_mesh* h) {
  std::vector<int> sds = h->sd_dirty;
  sds.insert(sds.end(), h->sd_always.begin(), h->sd_always.end());
  std::sort(sds.begin(), sds.end());
  sds.erase(std::unique(sds.begin(), sds.end()), sds.end());
  if (!h->j32_valid && h->opts.precision == HF_PREC_MIXED) convert_j32(h);
  factor_subdomains(h, sds);
  if (h->opts.coarse) {
    hf_status s = coarse_refactor(h);
    if (s) return s;
  }
  h->sd_dirty.clear();
  return check_cuda(h, cudaGetLastError(), "factor");
}

static void to_internal(const hf_mesh* h, const double* ext, std::vector<double>& in) {
  in.resize(h->N);
  int ned = h->ned;
  for (long long e = 0; e < h->ne; ++e)
    std::memcpy(&in[(size_t)h->ext2int[e] * ned], ext + e * ned, ned * sizeof(double));
  if (h->np) std::memcpy(&in[h->nu], ext + h->nu, h->np * sizeof(double));
}
static void to_external(const hf_mesh* h, const std::vector<double>& in, double* ext) {
  int ned = h->ned;
  for (long long e = 0; e < h->ne; ++e)
    std::memcpy(ext + e * ned, &in[(size_t)h->ext2int[e] * ned], ned * sizeof(double));
  if (h->np) std::memcpy(ext + h->nu, &in[h->nu], h->np * sizeof(double));
}

// ---------------------------------------------------------------- ABI
extern "C" {

void hf_default_solver_opts(hf_solver_opts* o) {
  if (!o) return;
  o->precision = HF_PREC_FP64;
  o->restart = 60;
  o->max_iters = 3000;
  o->rtol = 1e-12;
  o->inner_rtol = 1e-4;
  o->jacobi_block = 32;
  o->fluid_scaling = 1;
  o->newton_tol = 1e-10;
  o->use_graphs = 0;
  o->coarse = 1;
  o->coarse_max = 2048;
  o->reorth = 3;
  o->scheme = HF_SCHEME_COUPLED;
}

const char* hf_last_error(const hf_mesh* h) { return h ? h->err.c_str() : "null handle"; }

hf_status hf_get_sizes(const hf_mesh* h, int64_t* n_u, int64_t* n_p, int64_t* nfn) {
  if (!h) return HF_ERR_INVALID_ARG;
  if (n_u) *n_u = h->nu;
  if (n_p) *n_p = h->np;
  if (nfn) *nfn = h->nfn;
  return HF_OK;
}

hf_status hf_mesh_destroy(hf_mesh* h) {
  if (!h) return HF_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  invalidate_graphs(h);
  for (int i = 0; i < 2 * PROF_EVENTS; ++i)
    if (h->prof.ev[i]) cudaEventDestroy(h->prof.ev[i]);
  for (const hf_mesh::Alloc& a : h->allocs) cudaFreeAsync(a.raw, h->stream);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->prof.cyc_a) cudaEventDestroy(h->prof.cyc_a);
  if (h->prof.cyc_b) cudaEventDestroy(h->prof.cyc_b);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return HF_OK;
}

hf_status hf_mesh_create(const hf_mesh_desc* desc, void* cuda_stream, hf_mesh** out) {
  if (!desc || !out) return HF_ERR_INVALID_ARG;
  *out = nullptr;
  if ((desc->dim != 2 && desc->dim != 3) || desc->order != 2 || desc->n_nodes <= 0 || desc->n_elems <= 0 ||
      desc->n_faces <= 0 || !desc->xyz || !desc->elem_nodes || !desc->face_elems || !desc->face_local ||
      !desc->face_crackable || desc->n_elems > (1LL << 30) || desc->n_faces > (1LL << 30))
    return HF_ERR_INVALID_ARG;
  hf_mesh* h = new hf_mesh();
  const int dim = desc->dim;
  h->dim = dim;
  h->nen = dim == 2 ? 6 : 10;
  h->ned = h->nen * dim;
  h->nfn = dim == 2 ? 3 : 6;
  h->nfr = h->nfn * dim;
  h->ne = desc->n_elems;
  h->nf = desc->n_faces;
  h->nnodes = desc->n_nodes;
  hf_default_solver_opts(&h->opts);
  const int ne = (int)h->ne, nf = (int)h->nf, nen = h->nen, nsl = dim + 1, nfn = h->nfn;
  auto fail = [&](hf_status s, const std::string& msg) {
    h->err = msg;
    hf_mesh_destroy(h);
    return s;
  };
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(HF_ERR_CUDA, "cudaStreamCreate");
    h->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(HF_ERR_CUDA, "side stream of the preconditioner");
  // validate element nodes
  for (long long i = 0; i < (long long)ne * nen; ++i)
    if (desc->elem_nodes[i] < 0 || desc->elem_nodes[i] >= desc->n_nodes) return fail(HF_ERR_INVALID_ARG, "elem_nodes out of range");
  // Morton order of element centroids
  std::vector<double> lo(dim, 1e300), hi(dim, -1e300);
  for (long long g = 0; g < desc->n_nodes; ++g)
    for (int k = 0; k < dim; ++k) {
      lo[k] = std::min(lo[k], desc->xyz[g * dim + k]);
      hi[k] = std::max(hi[k], desc->xyz[g * dim + k]);
    }
  std::vector<std::pair<uint64_t, int>> key(ne);
  for (int e = 0; e < ne; ++e) {
    double c[3] = {0, 0, 0};
    for (int a = 0; a <= dim; ++a)
      for (int k = 0; k < dim; ++k) c[k] += desc->xyz[(long long)desc->elem_nodes[(long long)e * nen + a] * dim + k];
    uint64_t code = 0;
    for (int k = 0; k < dim; ++k) {
      double u = (c[k] / (dim + 1) - lo[k]) / std::max(hi[k] - lo[k], 1e-300);
      u = std::min(std::max(u, 0.0), 1.0);
      uint64_t qk = (uint64_t)(u * (dim == 2 ? 4294967295.0 : 2097151.0));
      code |= (dim == 2 ? spread2(qk) : spread3(qk)) << k;
    }
    key[e] = {code, e};
  }
  std::sort(key.begin(), key.end());
  h->int2ext.resize(ne);
  h->ext2int.resize(ne);
  for (int i = 0; i < ne; ++i) {
    h->int2ext[i] = key[i].second;
    h->ext2int[key[i].second] = i;
  }
  // element nodes (internal, SoA)
  std::vector<int> enode((size_t)nen * ne);
  for (int i = 0; i < ne; ++i)
    for (int a = 0; a < nen; ++a) enode[(size_t)a * ne + i] = desc->elem_nodes[(long long)h->int2ext[i] * nen + a];
  // facets
  h->h_fe.assign(2 * nf, -1);
  h->h_fl.assign(2 * nf, -1);
  h->h_crack.assign(nf, 0);
  std::vector<signed char> loc_m((size_t)nfn * nf, 0), loc_p((size_t)nfn * nf, 0);
  h->h_nbr.assign((size_t)nsl * ne, -1);
  h->h_slot_face.assign((size_t)nsl * ne, -1);
  h->h_slot_side.assign((size_t)nsl * ne, 0);
  for (int f = 0; f < nf; ++f) {
    int em = desc->face_elems[2 * f], ep = desc->face_elems[2 * f + 1];
    int jm = desc->face_local[2 * f], jp = desc->face_local[2 * f + 1];
    if (em < 0 || em >= ne || jm < 0 || jm > dim) return fail(HF_ERR_INVALID_ARG, "facet " + std::to_string(f) + ": bad e_minus");
    if (ep >= ne || (ep >= 0 && (jp < 0 || jp > dim))) return fail(HF_ERR_INVALID_ARG, "facet " + std::to_string(f) + ": bad e_plus");
    int im = h->ext2int[em];
    h->h_fe[f] = im;
    h->h_fl[f] = (signed char)jm;
    h->h_crack[f] = (ep >= 0 && desc->face_crackable[f]) ? 1 : 0;
    for (int a = 0; a < nfn; ++a) loc_m[(size_t)a * nf + f] = (signed char)fnode(dim, jm, a);
    if (h->h_slot_face[(size_t)jm * ne + im] >= 0) return fail(HF_ERR_INVALID_ARG, "two facets on one element side");
    h->h_slot_face[(size_t)jm * ne + im] = f;
    h->h_slot_side[(size_t)jm * ne + im] = 0;
    if (ep >= 0) {
      int ip = h->ext2int[ep];
      h->h_fe[nf + f] = ip;
      h->h_fl[nf + f] = (signed char)jp;
      // match face nodes of e_minus to local nodes of e_plus by global id
      for (int a = 0; a < nfn; ++a) {
        int g = desc->elem_nodes[(long long)em * nen + fnode(dim, jm, a)];
        int found = -1;
        for (int b = 0; b < nfn; ++b) {
          int lb = fnode(dim, jp, b);
          if (desc->elem_nodes[(long long)ep * nen + lb] == g) found = lb;
        }
        if (found < 0) return fail(HF_ERR_INVALID_ARG, "facet " + std::to_string(f) + ": elements do not share it");
        loc_p[(size_t)a * nf + f] = (signed char)found;
      }
      if (h->h_slot_face[(size_t)jp * ne + ip] >= 0) return fail(HF_ERR_INVALID_ARG, "two facets on one element side");
      h->h_slot_face[(size_t)jp * ne + ip] = f;
      h->h_slot_side[(size_t)jp * ne + ip] = 1;
      h->h_nbr[(size_t)jm * ne + im] = ip;
      h->h_nbr[(size_t)jp * ne + ip] = im;
    } else {
      for (int a = 0; a < nfn; ++a) loc_p[(size_t)a * nf + f] = loc_m[(size_t)a * nf + f];
    }
  }
  // pressure unknowns: nodes of crackable facets, ascending global id
  std::vector<int> pmap(desc->n_nodes, -1);
  for (int f = 0; f < nf; ++f) {
    if (!h->h_crack[f]) continue;
    int em = desc->face_elems[2 * f], jm = desc->face_local[2 * f];
    for (int a = 0; a < nfn; ++a) pmap[desc->elem_nodes[(long long)em * nen + fnode(dim, jm, a)]] = 1;
  }
  int np = 0;
  for (long long g = 0; g < desc->n_nodes; ++g)
    if (pmap[g] > 0) {
      pmap[g] = np++;
      h->p_nodes.push_back(g);
    }
  h->np = np;
  h->nu = (long long)ne * h->ned;
  h->N = h->nu + np;
  h->hp_fpdof.assign((size_t)nfn * nf, -1);
  std::vector<int> pcount(np + 1, 0);
  for (int f = 0; f < nf; ++f) {
    if (!h->h_crack[f]) continue;
    int em = desc->face_elems[2 * f], jm = desc->face_local[2 * f];
    for (int a = 0; a < nfn; ++a) {
      int pd = pmap[desc->elem_nodes[(long long)em * nen + fnode(dim, jm, a)]];
      h->hp_fpdof[(size_t)a * nf + f] = pd;
      pcount[pd + 1]++;
    }
  }
  for (int g = 0; g < np; ++g) pcount[g + 1] += pcount[g];
  std::vector<int> pinc_face(pcount[np]);
  std::vector<signed char> pinc_a(pcount[np]);
  {
    std::vector<int> fill(pcount.begin(), pcount.end() - 1);
    for (int f = 0; f < nf; ++f) {
      if (!h->h_crack[f]) continue;
      for (int a = 0; a < nfn; ++a) {
        int pd = h->hp_fpdof[(size_t)a * nf + f];
        pinc_face[fill[pd]] = f;
        pinc_a[fill[pd]++] = (signed char)a;
      }
    }
  }
  // Dirichlet rows and values
  std::vector<unsigned> dirmask(ne, 0);
  std::vector<double> ubar(h->nu, 0.0);
  for (long long i = 0; i < desc->n_dirichlet; ++i) {
    long long d = desc->dir_dof[i];
    if (d < 0 || d >= h->nu) return fail(HF_ERR_INVALID_ARG, "dir_dof out of range");
    int e = (int)(d / h->ned), r = (int)(d % h->ned);
    int ie = h->ext2int[e];
    dirmask[ie] |= 1u << r;
    ubar[(size_t)ie * h->ned + r] = desc->dir_val ? desc->dir_val[i] : 0.0;
  }
  // Neumann tractions per facet
  std::vector<double> ftrac((size_t)dim * nf, 0.0);
  std::vector<signed char> fneu(nf, 0);
  for (long long i = 0; i < desc->n_neumann; ++i) {
    int f = desc->neu_face[i];
    if (f < 0 || f >= nf || desc->face_elems[2 * f + 1] >= 0) return fail(HF_ERR_INVALID_ARG, "neu_face must be a boundary facet");
    fneu[f] = 1;
    for (int k = 0; k < dim; ++k) ftrac[(size_t)k * nf + f] = desc->neu_traction[i * dim + k];
  }
  // device copies
  DevMesh& d = h->d;
  d.dim = dim;
  d.nen = nen;
  d.ned = h->ned;
  d.nfn = nfn;
  d.nfr = h->nfr;
  d.nslot = nsl;
  d.ne = ne;
  d.nf = nf;
  d.np = np;
  d.nu = h->nu;
  d.N = h->N;
  std::vector<double> xyz(desc->xyz, desc->xyz + desc->n_nodes * dim);
  d.xyz = upload(h, xyz);
  d.enode = upload(h, enode);
  d.grad_lam = dzeros<double>(h, (size_t)(dim + 1) * dim * ne);
  d.vol = dzeros<double>(h, ne);
  d.nbr = upload(h, h->h_nbr);
  d.slot_face = upload(h, h->h_slot_face);
  d.slot_side = upload(h, h->h_slot_side);
  d.dirmask = upload(h, dirmask);
  d.nlmask = dzeros<unsigned char>(h, ne);
  d.fe = upload(h, h->h_fe);
  d.fl = upload(h, h->h_fl);
  d.fnormal = dzeros<double>(h, (size_t)dim * nf);
  d.farea = dzeros<double>(h, nf);
  d.fh = dzeros<double>(h, nf);
  d.fsg = dzeros<double>(h, (size_t)dim * dim * nf);
  d.loc_m = upload(h, loc_m);
  d.loc_p = upload(h, loc_p);
  d.fpdof = upload(h, h->hp_fpdof);
  d.crack = upload(h, h->h_crack);
  h->h_alpha.assign(nf, 0);
  h->h_beta.assign(nf, 0);
  d.alpha = dzeros<signed char>(h, nf);
  d.beta = dzeros<signed char>(h, nf);
  d.w_old = dzeros<double>(h, (size_t)nfn * nf);
  d.nl = dzeros<double>(h, (size_t)nf * (dim == 2 ? Shape<2>::nld : Shape<3>::nld));
  d.pinc_ptr = upload(h, pcount);
  d.pinc_face = upload(h, pinc_face);
  d.pinc_a = upload(h, pinc_a);
  d.p_active = dzeros<signed char>(h, np);
  d.inj_w = dzeros<double>(h, np);
  d.p_fixval = upload(h, std::vector<double>(std::max<size_t>(np, 1), std::nan("")));
  d.sinv_d = dzeros<double>(h, np);
  d.phase = 0;
  d.ubar = upload(h, ubar);
  d.fext = dzeros<double>(h, h->nu);
  d.scal = dzeros<double>(h, 16);
  d.err_flag = dzeros<int>(h, 4);
  d.wait_polls = 1 << 22;
  h->fneu_trac = upload(h, ftrac);
  h->fneu = upload(h, fneu);
  size_t nmat = (size_t)ne * (h->ned * h->ned + nsl * h->ned * h->nfr);
  h->J64.dg = dzeros<double>(h, nmat);
  h->J64.off = h->J64.dg ? h->J64.dg + (size_t)ne * h->ned * h->ned : nullptr;
  h->X = dzeros<double>(h, h->N);
  h->R = dzeros<double>(h, h->N);
  h->D = dzeros<double>(h, h->N);
  h->tmp64 = dzeros<double>(h, h->N);
  h->r64 = dzeros<double>(h, h->N);
  h->d_elist = dzeros<int>(h, ne);
  h->d_count = dzeros<int>(h, 16);
  h->d_red = dzeros<double>(h, 16);
  h->d_wtmp = dzeros<double>(h, (size_t)std::max(nfn, 1) * nf);
  if (!d.xyz || !d.enode || !d.grad_lam || !d.vol || !d.nbr || !d.slot_face || !d.slot_side || !d.dirmask ||
      !d.nlmask || !d.fe || !d.fl || !d.fnormal || !d.farea || !d.fh || !d.fsg || !d.loc_m || !d.loc_p ||
      !d.fpdof || !d.crack || !d.alpha || !d.beta || !d.w_old || !d.nl || !d.pinc_ptr || !d.pinc_face ||
      !d.pinc_a || !d.p_active || !d.inj_w || !d.p_fixval || !d.sinv_d || !d.ubar || !d.fext || !d.scal || !d.err_flag || !h->fneu_trac || !h->fneu ||
      !h->J64.dg || !h->X || !h->R || !h->D || !h->tmp64 || !h->r64 || !h->d_elist || !h->d_count ||
      !h->d_red || !h->d_wtmp)
    return fail(HF_ERR_OOM, "device allocation failed");
  build_quad(dim, h->q);
  if (build_subdomains(h, h->opts.jacobi_block)) return fail(HF_ERR_OOM, h->err);
  if (solver_alloc(h)) return fail(HF_ERR_OOM, h->err);
  if (dim == 2) launch_geometry<2>(d, h->stream);
  else launch_geometry<3>(d, h->stream);
  if (coarse_layout(h)) return fail(HF_ERR_OOM, h->err);
  double one = 1.0;
  cudaMemcpyAsync(d.scal, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HF_ERR_CUDA, std::string("mesh set-up: ") + cudaGetErrorString(e));
  *out = h;
  return HF_OK;
}

hf_status hf_set_material(hf_mesh* h, double E, double nu, double sigma_c, double delta_c, double b_stab) {
  HF_GUARD(h);
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(sigma_c > 0) || !(delta_c > 0) || !(b_stab > 0))
    return set_error(h, HF_ERR_INVALID_ARG, "material parameters out of range");
  h->E = E;
  h->nu_p = nu;
  h->sigma_c = sigma_c;
  h->delta_c = delta_c;
  h->b_stab = b_stab;
  h->d.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  h->d.mu = E / (2.0 * (1.0 + nu));
  h->d.sigma_c = sigma_c;
  h->d.delta_c = delta_c;
  h->d.b_stab = b_stab;
  h->material_set = true;
  invalidate_graphs(h);
  cudaMemsetAsync(h->d.fext, 0, h->nu * sizeof(double), h->stream);
  if (h->dim == 2) launch_neumann<2>(h->d, h->q, h->fneu_trac, h->fneu, h->stream);
  else launch_neumann<3>(h->d, h->q, h->fneu_trac, h->fneu, h->stream);
  std::vector<int> all(h->ne);
  std::iota(all.begin(), all.end(), 0);
  hf_status s = rebuild_rows(h, all);
  if (s) return s;
  h->sd_dirty = all_subdomains(h);
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set_material");
}

hf_status hf_set_injection(hf_mesh* h, double mu, double Q0, int64_t n_inj, const int64_t* p_dofs,
                           const double* weights, double delta_f, double dt, double p_vapor, int cutoff_on,
                           double L_ref) {
  HF_GUARD(h);
  if (!(mu > 0) || !(dt > 0) || !(delta_f >= 0) || !(L_ref > 0) || n_inj < 0 || (n_inj > 0 && !p_dofs))
    return set_error(h, HF_ERR_INVALID_ARG, "injection parameters out of range");
  std::vector<double> w(h->np, 0.0);
  for (int64_t i = 0; i < n_inj; ++i) {
    if (p_dofs[i] < 0 || p_dofs[i] >= h->np) return set_error(h, HF_ERR_INVALID_ARG, "injection dof out of range");
    w[p_dofs[i]] += weights ? weights[i] : 1.0;
  }
  h->mu_f = mu;
  h->Q0 = Q0;
  h->delta_f = delta_f;
  h->dt = dt;
  h->p_v = p_vapor;
  h->cutoff = cutoff_on ? 1 : 0;
  h->L_ref = L_ref;
  h->d.mu_f = mu;
  h->d.Q0 = Q0;
  h->d.delta_f = delta_f;
  h->d.dt = dt;
  h->d.p_v = p_vapor;
  h->d.cutoff = h->cutoff;
  if (h->np) cudaMemcpyAsync(h->d.inj_w, w.data(), h->np * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  launch_fluid_scale(h->d, h->opts.fluid_scaling, h->L_ref, h->stream);
  h->injection_set = true;
  invalidate_graphs(h);
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set_injection");
}

hf_status hf_set_solver(hf_mesh* h, const hf_solver_opts* o) {
  HF_GUARD(h);
  if (!o || (o->precision != HF_PREC_FP64 && o->precision != HF_PREC_MIXED) || o->restart < 1 || o->restart > GM_MAX ||
      o->max_iters < 0 || !(o->rtol > 0) || !(o->inner_rtol > 0) || o->jacobi_block < 1 || o->coarse < 0 ||
      o->coarse > 1 || o->coarse_max < 16 || o->coarse_max > 4096 || o->reorth < 0 || o->reorth > 3 ||
      (o->scheme != HF_SCHEME_COUPLED && o->scheme != HF_SCHEME_STAGGERED) ||
      (o->scheme == HF_SCHEME_STAGGERED && o->precision != HF_PREC_FP64))
    return set_error(h, HF_ERR_INVALID_ARG, "solver options out of range");
  bool regroup = std::min(256, o->jacobi_block) != h->G;
  bool rescale = o->fluid_scaling != h->opts.fluid_scaling;
  bool relayout = o->coarse_max != h->opts.coarse_max || o->coarse != h->opts.coarse;
  h->opts = *o;
  invalidate_graphs(h);
  {
    hf_status s = krylov_basis_alloc(h, o->restart);
    if (s) return s;
  }
  if (relayout) {
    hf_status s = coarse_layout(h);
    if (s) return s;
  }
  if (regroup) {
    hf_status s = build_subdomains(h, o->jacobi_block);
    if (s) return s;
    rebuild_lists(h);
  }
  h->sd_dirty = all_subdomains(h);
  if (rescale && h->injection_set) launch_fluid_scale(h->d, h->opts.fluid_scaling, h->L_ref, h->stream);
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set_solver");
}

hf_status hf_set_state(hf_mesh* h, const double* U, const double* P, const int8_t* alpha, const int8_t* beta,
                       const double* w_old, double t) {
  HF_GUARD(h);
  if (!h->material_set || !h->injection_set) return set_error(h, HF_ERR_STATE, "set material and injection first");
  if (!U || (h->np && !P) || !alpha || !beta) return set_error(h, HF_ERR_INVALID_ARG, "null state array");
  std::vector<double> ext(h->N), in;
  std::memcpy(ext.data(), U, h->nu * sizeof(double));
  if (h->np) std::memcpy(ext.data() + h->nu, P, h->np * sizeof(double));
  to_internal(h, ext.data(), in);
  HF_CUDA(h, cudaMemcpyAsync(h->X, in.data(), h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  std::vector<int> changed;
  for (long long f = 0; f < h->nf; ++f) {
    signed char a = h->h_crack[f] ? (alpha[f] ? 1 : 0) : 0;
    signed char b = h->h_crack[f] ? (beta[f] ? 1 : 0) : 0;
    if (a != h->h_alpha[f]) {
      changed.push_back(h->h_fe[f]);
      if (h->h_fe[h->nf + f] >= 0) changed.push_back(h->h_fe[h->nf + f]);
    }
    h->h_alpha[f] = a;
    h->h_beta[f] = b;
  }
  hf_status s = rebuild_lists(h);
  if (s) return s;
  std::sort(changed.begin(), changed.end());
  changed.erase(std::unique(changed.begin(), changed.end()), changed.end());
  if ((s = rebuild_rows(h, changed))) return s;
  if (w_old) {
    std::vector<double> wo((size_t)h->nfn * h->nf);
    for (long long f = 0; f < h->nf; ++f)
      for (int a = 0; a < h->nfn; ++a) wo[(size_t)a * h->nf + f] = w_old[f * h->nfn + a];
    HF_CUDA(h, cudaMemcpyAsync(h->d.w_old, wo.data(), wo.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  } else {
    if (h->dim == 2) launch_openings<2>(h->d, h->X, h->d.w_old, h->stream);
    else launch_openings<3>(h->d, h->X, h->d.w_old, h->stream);
  }
  launch_fluid_scale(h->d, h->opts.fluid_scaling, h->L_ref, h->stream);
  h->t = t;
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set_state");
}

hf_status hf_get_state(hf_mesh* h, double* U, double* P, int8_t* alpha, int8_t* beta, double* w_old, double* t) {
  HF_GUARD(h);
  std::vector<double> in(h->N), ext(h->N);
  HF_CUDA(h, cudaMemcpyAsync(in.data(), h->X, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> wo((size_t)h->nfn * h->nf);
  HF_CUDA(h, cudaMemcpyAsync(wo.data(), h->d.w_old, wo.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  to_external(h, in, ext.data());
  if (U) std::memcpy(U, ext.data(), h->nu * sizeof(double));
  if (P && h->np) std::memcpy(P, ext.data() + h->nu, h->np * sizeof(double));
  if (alpha) for (long long f = 0; f < h->nf; ++f) alpha[f] = h->h_alpha[f];
  if (beta) for (long long f = 0; f < h->nf; ++f) beta[f] = h->h_beta[f];
  if (w_old)
    for (long long f = 0; f < h->nf; ++f)
      for (int a = 0; a < h->nfn; ++a) w_old[f * h->nfn + a] = wo[(size_t)a * h->nf + f];
  if (t) *t = h->t;
  return HF_OK;
}

static hf_status assemble_nl(hf_mesh* h) {
  prof_begin(h, PK_ASSEMBLY);
  if (h->dim == 2) launch_face_nl<2>(h->d, h->q, h->X, h->stream);
  else launch_face_nl<3>(h->d, h->q, h->X, h->stream);
  prof_end(h);
  return check_cuda(h, cudaGetLastError(), "face_nl");
}

// One iteration of the staggered scheme (Sec. 4.3): the mechanical equation
// solved for U with the pressure of the previous iteration, A dU = -R_u(U, P),
// then the lubrication equation for P at the new opening, D dP =
// -R_p(U + dU, P).  Both solves use the GMRES of the coupled system with the
// other block's rows turned into identity rows (DevMesh::phase).
static hf_status staggered_step(hf_mesh* h, hf_newton_report* rep) {
  hf_newton_report r{}, r1{}, r2{};
  hf_status s;
  double n1[4], n2[4];
  if ((s = assemble_nl(h))) return s;
  residual(h, h->X, h->R);
  r.res_norm = sqrt(device_norm2(h, h->R, h->N));
  if (!std::isfinite(r.res_norm)) return set_error(h, HF_ERR_NONFINITE, "residual is not finite");
  if ((s = refactor(h))) return s;
  launch_neg_part(h, h->R, h->K64.b, 1, 0);
  h->d.phase = 1;
  s = linear_solve(h, h->K64.b, h->D, &r1);
  h->d.phase = 0;
  if (s) return s;
  if ((s = newton_update(h, h->D, n1))) return s;
  if ((s = assemble_nl(h))) return s;
  residual(h, h->X, h->R);
  launch_neg_part(h, h->R, h->K64.b, 0, 1);
  launch_diag_d(h);
  h->d.phase = 2;
  s = linear_solve(h, h->K64.b, h->D, &r2);
  h->d.phase = 0;
  if (s) return s;
  if ((s = newton_update(h, h->D, n2))) return s;
  r.du_rel = sqrt(n1[0]) / std::max(sqrt(n1[1]), 1e-300);
  r.dp_rel = h->np ? sqrt(n2[2]) / std::max(sqrt(n2[3]), 1e-300) : 0.0;
  r.gmres_iters = r1.gmres_iters + r2.gmres_iters;
  r.lin_res = std::max(r1.lin_res, r2.lin_res);
  r.lin_converged = r1.lin_converged && r2.lin_converged;
  if (!std::isfinite(r.du_rel) || !std::isfinite(r.dp_rel)) return set_error(h, HF_ERR_NONFINITE, "update is not finite");
  r.converged = r.du_rel <= h->opts.newton_tol && r.dp_rel <= h->opts.newton_tol;
  if (rep) *rep = r;
  return HF_OK;
}

hf_status hf_set_fixed_pressure(hf_mesh* h, int64_t n, const int64_t* p_dofs, const double* values) {
  HF_GUARD(h);
  if (n < 0 || (n > 0 && (!p_dofs || !values))) return set_error(h, HF_ERR_INVALID_ARG, "null fixed-pressure arrays");
  std::vector<double> v(std::max<long long>(h->np, 1), std::nan(""));
  for (int64_t i = 0; i < n; ++i) {
    if (p_dofs[i] < 0 || p_dofs[i] >= h->np) return set_error(h, HF_ERR_INVALID_ARG, "fixed pressure dof out of range");
    if (!std::isfinite(values[i])) return set_error(h, HF_ERR_INVALID_ARG, "fixed pressure value not finite");
    v[p_dofs[i]] = values[i];
  }
  HF_CUDA(h, cudaMemcpyAsync(h->d.p_fixval, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->sd_dirty = all_subdomains(h);
  invalidate_graphs(h);
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set_fixed_pressure");
}

hf_status hf_set_wait_limit(hf_mesh* h, int64_t polls) {
  HF_GUARD(h);
  if (polls < 1 || polls > (int64_t)1 << 30) return set_error(h, HF_ERR_INVALID_ARG, "wait limit out of range");
  h->d.wait_polls = (int)polls;
  invalidate_graphs(h);
  return HF_OK;
}

hf_status hf_check_wait_timeout(hf_mesh* h) {
  HF_GUARD(h);
  HF_CUDA(h, cudaMemsetAsync(h->d.err_flag, 0, sizeof(int), h->stream));
  launch_wait_selftest(h);
  int flag = 0;
  HF_CUDA(h, cudaMemcpyAsync(&flag, h->d.err_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (flag) {
    HF_CUDA(h, cudaMemsetAsync(h->d.err_flag, 0, sizeof(int), h->stream));
    HF_CUDA(h, cudaStreamSynchronize(h->stream));
    return set_error(h, HF_ERR_TIMEOUT, "a bounded device wait timed out (self-test barrier)");
  }
  return HF_OK;
}

hf_status hf_newton_step(hf_mesh* h, hf_newton_report* rep) {
  HF_GUARD(h);
  if (!h->material_set || !h->injection_set) return set_error(h, HF_ERR_STATE, "set material and injection first");
  if (h->opts.scheme == HF_SCHEME_STAGGERED) return staggered_step(h, rep);
  hf_newton_report r{};
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  residual(h, h->X, h->R);
  double rn2 = device_norm2(h, h->R, h->N);
  r.res_norm = sqrt(rn2);
  if (!std::isfinite(r.res_norm)) return set_error(h, HF_ERR_NONFINITE, "residual is not finite");
  if ((s = refactor(h))) return s;
  launch_neg(h, h->R, h->tmp64);
  // the solve may use tmp64 as scratch: keep -R in K64.b
  cudaMemcpyAsync(h->K64.b, h->tmp64, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  if ((s = linear_solve(h, h->K64.b, h->D, &r))) return s;
  double nrm[4];
  if ((s = newton_update(h, h->D, nrm))) return s;
  r.du_rel = sqrt(nrm[0]) / std::max(sqrt(nrm[1]), 1e-300);
  r.dp_rel = h->np ? sqrt(nrm[2]) / std::max(sqrt(nrm[3]), 1e-300) : 0.0;
  if (!std::isfinite(r.du_rel) || !std::isfinite(r.dp_rel)) return set_error(h, HF_ERR_NONFINITE, "update is not finite");
  r.converged = r.du_rel <= h->opts.newton_tol && r.dp_rel <= h->opts.newton_tol;
  if (rep) *rep = r;
  return HF_OK;
}

hf_status hf_check_fracture_criterion(hf_mesh* h, int64_t* n_new_alpha) {
  HF_GUARD(h);
  HF_CUDA(h, cudaMemsetAsync(h->d_count, 0, sizeof(int), h->stream));
  if (h->dim == 2) launch_criterion<2>(h->d, h->q, h->X, nullptr, h->d_count, h->stream);
  else launch_criterion<3>(h->d, h->q, h->X, nullptr, h->d_count, h->stream);
  int cnt = 0;
  HF_CUDA(h, cudaMemcpyAsync(&cnt, h->d_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (cnt > 0) {
    std::vector<signed char> a(h->nf);
    HF_CUDA(h, cudaMemcpyAsync(a.data(), h->d.alpha, h->nf, cudaMemcpyDeviceToHost, h->stream));
    HF_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int> changed;
    for (long long f = 0; f < h->nf; ++f)
      if (a[f] != h->h_alpha[f]) {
        h->h_alpha[f] = a[f];
        changed.push_back(h->h_fe[f]);
        if (h->h_fe[h->nf + f] >= 0) changed.push_back(h->h_fe[h->nf + f]);
      }
    hf_status s;
    if ((s = rebuild_lists(h))) return s;
    std::sort(changed.begin(), changed.end());
    changed.erase(std::unique(changed.begin(), changed.end()), changed.end());
    if ((s = rebuild_rows(h, changed))) return s;
  }
  if (n_new_alpha) *n_new_alpha = cnt;
  return check_cuda(h, cudaStreamSynchronize(h->stream), "criterion");
}

hf_status hf_accept_step(hf_mesh* h, int64_t* n_new_beta) {
  HF_GUARD(h);
  HF_CUDA(h, cudaMemsetAsync(h->d_count + 1, 0, sizeof(int), h->stream));
  if (h->dim == 2) launch_accept<2>(h->d, h->q, h->X, h->d_count + 1, h->stream);
  else launch_accept<3>(h->d, h->q, h->X, h->d_count + 1, h->stream);
  launch_fluid_scale(h->d, h->opts.fluid_scaling, h->L_ref, h->stream);
  int cnt = 0;
  HF_CUDA(h, cudaMemcpyAsync(&cnt, h->d_count + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (cnt > 0) {
    std::vector<signed char> b(h->nf);
    HF_CUDA(h, cudaMemcpyAsync(b.data(), h->d.beta, h->nf, cudaMemcpyDeviceToHost, h->stream));
    HF_CUDA(h, cudaStreamSynchronize(h->stream));
    for (long long f = 0; f < h->nf; ++f) h->h_beta[f] = b[f];
    hf_status s;
    if ((s = rebuild_lists(h))) return s;
  }
  h->t += h->dt;
  if (n_new_beta) *n_new_beta = cnt;
  return check_cuda(h, cudaStreamSynchronize(h->stream), "accept");
}

// ---------------------------------------------------------------- time step
// Start-of-step state kept on the device, so a failed attempt is undone
// without a host round trip.
static hf_status snap_save(hf_mesh* h) {
  if (!h->snap_X) {
    h->snap_X = static_cast<double*>(dev_alloc(h, h->N * sizeof(double)));
    h->snap_wold = static_cast<double*>(dev_alloc(h, (size_t)h->nfn * h->nf * sizeof(double)));
    if (!h->snap_X || !h->snap_wold) return set_error(h, HF_ERR_OOM, "step snapshot");
  }
  HF_CUDA(h, cudaMemcpyAsync(h->snap_X, h->X, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  HF_CUDA(h, cudaMemcpyAsync(h->snap_wold, h->d.w_old, (size_t)h->nfn * h->nf * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  h->snap_alpha = h->h_alpha;
  h->snap_beta = h->h_beta;
  h->snap_t = h->t;
  return HF_OK;
}

static hf_status snap_restore(hf_mesh* h) {
  HF_CUDA(h, cudaMemcpyAsync(h->X, h->snap_X, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  HF_CUDA(h, cudaMemcpyAsync(h->d.w_old, h->snap_wold, (size_t)h->nfn * h->nf * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  std::vector<int> changed;
  for (long long f = 0; f < h->nf; ++f)
    if (h->h_alpha[f] != h->snap_alpha[f]) {
      changed.push_back(h->h_fe[f]);
      if (h->h_fe[h->nf + f] >= 0) changed.push_back(h->h_fe[h->nf + f]);
    }
  h->h_alpha = h->snap_alpha;
  h->h_beta = h->snap_beta;
  h->t = h->snap_t;
  hf_status s = rebuild_lists(h);
  if (s) return s;
  std::sort(changed.begin(), changed.end());
  changed.erase(std::unique(changed.begin(), changed.end()), changed.end());
  if ((s = rebuild_rows(h, changed))) return s;
  launch_fluid_scale(h->d, h->opts.fluid_scaling, h->L_ref, h->stream);
  return check_cuda(h, cudaGetLastError(), "restore");
}

// attempts (accepted sub-steps and failures) one hf_advance_step may take
constexpr int HF_STEP_MAX_ATTEMPTS = 256;

// the time-step length enters the facet records and the pressure rows, both
// baked into captured GMRES cycles
static void set_dt(hf_mesh* h, double dt) {
  if (dt == h->dt) return;
  h->dt = dt;
  h->d.dt = dt;
  invalidate_graphs(h);
}

static bool fatal(hf_mesh* h, hf_status s) {
  return h->poisoned || s == HF_ERR_CUDA || s == HF_ERR_TIMEOUT || s == HF_ERR_DEVICE_ASSERT || s == HF_ERR_OOM ||
         s == HF_ERR_INVALID_ARG || s == HF_ERR_STATE;
}

hf_status hf_get_opening_pressure(hf_mesh* h, double* w_face_nodes, double* p, int8_t* alpha, int8_t* beta) {
  HF_GUARD(h);
  if (w_face_nodes) {
    if (h->dim == 2) launch_openings<2>(h->d, h->X, h->d_wtmp, h->stream);
    else launch_openings<3>(h->d, h->X, h->d_wtmp, h->stream);
    std::vector<double> w((size_t)h->nfn * h->nf);
    HF_CUDA(h, cudaMemcpyAsync(w.data(), h->d_wtmp, w.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HF_CUDA(h, cudaStreamSynchronize(h->stream));
    for (long long f = 0; f < h->nf; ++f)
      for (int a = 0; a < h->nfn; ++a) w_face_nodes[f * h->nfn + a] = w[(size_t)a * h->nf + f];
  }
  if (p && h->np) {
    HF_CUDA(h, cudaMemcpyAsync(p, h->X + h->nu, h->np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HF_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (alpha) for (long long f = 0; f < h->nf; ++f) alpha[f] = h->h_alpha[f];
  if (beta) for (long long f = 0; f < h->nf; ++f) beta[f] = h->h_beta[f];
  return HF_OK;
}

hf_status hf_eval_residual(hf_mesh* h, double* Rout) {
  HF_GUARD(h);
  if (!Rout) return HF_ERR_INVALID_ARG;
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  residual(h, h->X, h->R);
  std::vector<double> in(h->N);
  HF_CUDA(h, cudaMemcpyAsync(in.data(), h->R, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  to_external(h, in, Rout);
  return HF_OK;
}

hf_status hf_apply_jacobian(hf_mesh* h, const double* x, double* y) {
  HF_GUARD(h);
  if (!x || !y) return HF_ERR_INVALID_ARG;
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  std::vector<double> in;
  to_internal(h, x, in);
  HF_CUDA(h, cudaMemcpyAsync(h->tmp64, in.data(), h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  apply_jacobian(h, h->tmp64, h->r64);
  HF_CUDA(h, cudaMemcpyAsync(in.data(), h->r64, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  to_external(h, in, y);
  return HF_OK;
}

hf_status hf_get_criterion_traction(hf_mesh* h, double* tmax) {
  HF_GUARD(h);
  if (!tmax) return HF_ERR_INVALID_ARG;
  if (h->dim == 2) launch_criterion<2>(h->d, h->q, h->X, h->d_wtmp, nullptr, h->stream);
  else launch_criterion<3>(h->d, h->q, h->X, h->d_wtmp, nullptr, h->stream);
  HF_CUDA(h, cudaMemcpyAsync(tmax, h->d_wtmp, h->nf * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_cuda(h, cudaStreamSynchronize(h->stream), "criterion traction");
}

hf_status hf_solve_linear(hf_mesh* h, const double* rhs, double* dsol, hf_newton_report* rep) {
  HF_GUARD(h);
  if (!rhs || !dsol) return HF_ERR_INVALID_ARG;
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  if ((s = refactor(h))) return s;
  std::vector<double> in;
  to_internal(h, rhs, in);
  HF_CUDA(h, cudaMemcpyAsync(h->K64.b, in.data(), h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  hf_newton_report r{};
  if ((s = linear_solve(h, h->K64.b, h->D, &r))) return s;
  HF_CUDA(h, cudaMemcpyAsync(in.data(), h->D, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  to_external(h, in, dsol);
  if (rep) *rep = r;
  return HF_OK;
}

hf_status hf_apply_preconditioner(hf_mesh* h, const double* x, double* z) {
  HF_GUARD(h);
  if (!x || !z) return HF_ERR_INVALID_ARG;
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  if ((s = refactor(h))) return s;
  std::vector<double> in;
  to_internal(h, x, in);
  HF_CUDA(h, cudaMemcpyAsync(h->tmp64, in.data(), h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  launch_precond64(h, h->tmp64, h->r64);
  HF_CUDA(h, cudaMemcpyAsync(in.data(), h->r64, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  to_external(h, in, z);
  return HF_OK;
}

hf_status hf_set_profiling(hf_mesh* h, int on) {
  HF_GUARD(h);
  if (on < 0 || on > 2) return set_error(h, HF_ERR_INVALID_ARG, "profiling mode out of range");
  prof_flush(h);
  h->prof.on = on == 1;
  h->prof.cycles = on == 2;
  if (on == 2 && !h->prof.cyc_a) {
    HF_CUDA(h, cudaEventCreate(&h->prof.cyc_a));
    HF_CUDA(h, cudaEventCreate(&h->prof.cyc_b));
  }
  for (int k = 0; k < PK_COUNT; ++k) {
    h->prof.ms[k] = 0.0;
    h->prof.launches[k] = 0;
  }
  h->prof.cycle_ms = 0.0;
  h->prof.cycle_steps = 0;
  return HF_OK;
}

hf_status hf_get_kernel_times(hf_mesh* h, double* ms, int64_t* launches) {
  HF_GUARD(h);
  HF_CUDA(h, cudaStreamSynchronize(h->stream));
  prof_flush(h);
  for (int k = 0; k < PK_COUNT; ++k) {
    if (ms) ms[k] = h->prof.ms[k];
    if (launches) launches[k] = h->prof.launches[k];
  }
  if (ms) ms[PK_COUNT] = h->prof.cycle_ms;
  if (launches) launches[PK_COUNT] = h->prof.cycle_steps;
  return HF_OK;
}

hf_status hf_get_stats(const hf_mesh* h, int64_t* st) {
  if (!h || !st) return HF_ERR_INVALID_ARG;
  st[0] = h->ne;
  st[1] = h->n_interior_slots;
  st[2] = h->n_subdomain_slots;
  st[3] = h->levels_max;
  st[4] = h->d.nsd;
  st[5] = h->d.n_nl;
  st[6] = h->np;
  st[7] = h->nf;
  st[8] = total_launches();
  st[9] = h->prof.graph_timing_error;
  st[10] = h->bytes_allocated;
  st[11] = h->opts.coarse ? h->nc : 0;
  st[12] = h->agg_size;
  st[13] = h->gs_reorths;
  st[14] = h->gs_cols;
  st[15] = h->gs_reorth_cols;
  return HF_OK;
}

void hf_default_step_opts(hf_step_opts* o) {
  if (!o) return;
  o->newton_max = 8;
  o->criterion_rounds = 4;
  o->max_cutbacks = 10;
  o->max_new_facets = 0;
}

hf_status hf_advance_step(hf_mesh* h, const hf_step_opts* opts, hf_step_report* rep) {
  HF_GUARD(h);
  if (!h->material_set || !h->injection_set) return set_error(h, HF_ERR_STATE, "set material and injection first");
  hf_step_opts o;
  hf_default_step_opts(&o);
  if (opts) o = *opts;
  if (o.newton_max < 1 || o.criterion_rounds < 1 || o.max_cutbacks < 0 || o.max_new_facets < 0)
    return set_error(h, HF_ERR_INVALID_ARG, "step options out of range");
  hf_step_report r{};
  const double dt0 = h->dt, target = h->t + dt0;
  double sub = dt0;
  int cuts = 0;         // consecutive failed attempts
  int attempts = 0;
  hf_status s = snap_save(h);
  if (s) return s;
  while (target - h->t > 1e-12 * dt0) {
    sub = std::min(sub, target - h->t);
    set_dt(h, sub);
    bool ok = false;
    int rounds = 0, it = 0;
    double prev_inc = HUGE_VAL;  // largest relative increment of the previous iteration
    for (;;) {  // Newton to convergence, then the criterion; Newton again if it switched facets
      hf_newton_report nr{};
      s = hf_newton_step(h, &nr);
      if (s != HF_OK) {
        if (fatal(h, s)) {
          set_dt(h, dt0);
          return s;
        }
        break;
      }
      ++r.newton_iters;
      r.gmres_iters += nr.gmres_iters;
      r.du_rel = nr.du_rel;
      r.dp_rel = nr.dp_rel;
      ++it;
      // a linear solve that stagnated within a decade of its tolerance (FP64
      // GMRES at its attainable accuracy) is accepted; one further off fails
      // the attempt
      if (!nr.lin_converged && !(nr.lin_res <= 10.0 * h->opts.rtol)) break;
      if (nr.converged) {
        int64_t na = 0;
        if ((s = hf_check_fracture_criterion(h, &na))) {
          set_dt(h, dt0);
          return s;
        }
        r.new_alpha += na;
        // a whole region switched at once: the sub-step overshot
        if (o.max_new_facets > 0 && na > o.max_new_facets) break;
        if (na == 0 || ++rounds >= o.criterion_rounds) {
          ok = true;
          break;
        }
        it = 0;
        prev_inc = HUGE_VAL;
        continue;
      }
      // past newton_max, keep going only while the increments still at least
      // halve every iteration (linear convergence), up to 4 newton_max
      const double inc = std::max(nr.du_rel, nr.dp_rel);
      if (it >= o.newton_max && (it >= 4 * o.newton_max || !(inc <= 0.5 * prev_inc))) break;
      prev_inc = inc;
    }
    ++attempts;
    if (ok) {
      int64_t nb = 0;
      if ((s = hf_accept_step(h, &nb))) {
        set_dt(h, dt0);
        return s;
      }
      r.new_beta += nb;
      ++r.substeps;
      cuts = 0;
      if ((s = snap_save(h))) return s;
      sub = std::min(dt0, 1.5 * sub);
    } else {
      if ((s = snap_restore(h))) return s;
      if (++cuts > o.max_cutbacks || attempts >= HF_STEP_MAX_ATTEMPTS) {
        set_dt(h, dt0);
        if (rep) *rep = r;
        return set_error(h, HF_ERR_NOT_CONVERGED, "time step not converged after the allowed cutbacks");
      }
      ++r.cutbacks;
      sub *= 0.5;
    }
  }
  h->t = target;
  set_dt(h, dt0);
  r.t = h->t;
  if (rep) *rep = r;
  return check_cuda(h, cudaStreamSynchronize(h->stream), "advance_step");
}

// pressure unknowns (distinct nodes of crackable interior facets) and the
// number of crackable interior facets, from the descriptor alone
static hf_status desc_counts(const hf_mesh_desc* desc, long long* np_out, long long* ncrack_out) {
  if (!desc || (desc->dim != 2 && desc->dim != 3) || desc->n_elems <= 0 || desc->n_faces <= 0 ||
      desc->n_nodes <= 0 || !desc->elem_nodes || !desc->face_elems || !desc->face_local || !desc->face_crackable)
    return HF_ERR_INVALID_ARG;
  const long long dim = desc->dim, ne = desc->n_elems, nf = desc->n_faces, nn = desc->n_nodes;
  const long long nen = dim == 2 ? 6 : 10, nfn = dim == 2 ? 3 : 6;
  std::vector<char> mark(nn, 0);
  long long ncrack = 0;
  for (long long f = 0; f < nf; ++f) {
    int em = desc->face_elems[2 * f], ep = desc->face_elems[2 * f + 1], jm = desc->face_local[2 * f];
    if (ep < 0 || !desc->face_crackable[f] || em < 0 || em >= ne || jm < 0 || jm > dim) continue;
    ++ncrack;
    for (int a = 0; a < nfn; ++a) {
      int g = desc->elem_nodes[(long long)em * nen + fnode((int)dim, jm, a)];
      if (g >= 0 && g < nn) mark[g] = 1;
    }
  }
  long long np = 0;
  for (long long g = 0; g < nn; ++g) np += mark[g];
  *np_out = np;
  *ncrack_out = ncrack;
  return HF_OK;
}

hf_status hf_get_subdomains(const hf_mesh* h, int32_t* sd_of_elem, int32_t* order_in_sd) {
  if (!h) return HF_ERR_INVALID_ARG;
  for (long long e = 0; e < h->ne; ++e) {
    const int i = h->ext2int[e];
    if (sd_of_elem) sd_of_elem[e] = i / h->G;
    if (order_in_sd) order_in_sd[e] = i % h->G;
  }
  return HF_OK;
}

hf_status hf_get_aggregates(const hf_mesh* h, int32_t* agg_of_elem) {
  if (!h || !agg_of_elem || h->agg_size < 1) return HF_ERR_INVALID_ARG;
  for (long long e = 0; e < h->ne; ++e) agg_of_elem[e] = h->ext2int[e] / h->agg_size;
  return HF_OK;
}

hf_status hf_get_coarse_operator(hf_mesh* h, int64_t* nc, double* A0, double* A0inv, double* geo) {
  HF_GUARD(h);
  if (nc) *nc = h->opts.coarse ? h->nc : 0;
  if (!A0 && !A0inv && !geo) return HF_OK;
  hf_status s;
  if ((s = assemble_nl(h))) return s;
  if ((s = refactor(h))) return s;
  return coarse_rebuild_copy(h, A0, A0inv, geo);
}

hf_status hf_mesh_sizes(const hf_mesh_desc* desc, int64_t* n_u, int64_t* n_p) {
  long long np = 0, ncrack = 0;
  hf_status s = desc_counts(desc, &np, &ncrack);
  if (s) return s;
  if (n_u) *n_u = desc->n_elems * (desc->dim == 2 ? 12 : 30);
  if (n_p) *n_p = np;
  return HF_OK;
}

hf_status hf_estimate_device_bytes(const hf_mesh_desc* desc, const hf_solver_opts* opts, int64_t* bytes) {
  long long np = 0, ncrack = 0;
  if (!bytes || desc_counts(desc, &np, &ncrack) != HF_OK) return HF_ERR_INVALID_ARG;
  hf_solver_opts o;
  hf_default_solver_opts(&o);
  if (opts) o = *opts;
  const int jacobi_block = o.jacobi_block;
  // the bases are sized for the longest cycle the handle has been given: the
  // default at creation, then this one
  hf_solver_opts dflt;
  hf_default_solver_opts(&dflt);
  const long long mres = std::max(1, std::min(GM_MAX, std::max(o.restart, dflt.restart)));
  const long long dim = desc->dim, ne = desc->n_elems, nf = desc->n_faces, nn = desc->n_nodes;
  const long long nen = dim == 2 ? 6 : 10, ned = nen * dim, nfn = dim == 2 ? 3 : 6, nfr = nfn * dim, nsl = dim + 1;
  const long long nld = 4 * nfn * nfn + 3 * nfn, lus = ned * ned + nsl * ned * nfr;
  const long long nu = ne * ned, N = nu + np;
  const long long G = std::max(1, std::min(jacobi_block, 256)), nsd = (ne + G - 1) / G;
  const long long nmat = ne * (ned * ned + nsl * ned * nfr), ldv = (N + 63) / 64 * 64;
  long long t = 0;
  auto add = [&](long long b) { t += (std::max(b, 1LL) + 255) / 256 * 256; };
  // mesh arrays
  add(nn * dim * 8); add(nen * ne * 4); add((dim + 1) * dim * ne * 8); add(ne * 8);
  add(nsl * ne * 4); add(nsl * ne * 4); add(nsl * ne); add(ne * 4); add(ne);
  add(2 * nf * 4); add(2 * nf); add(dim * nf * 8); add(nf * 8); add(nf * 8); add(dim * dim * nf * 8);
  add(nfn * nf); add(nfn * nf); add(nfn * nf * 4); add(nf); add(nf); add(nf); add(nfn * nf * 8);
  add(nf * nld * 8); add((np + 1) * 4); add(ncrack * nfn * 4); add(ncrack * nfn); add(np); add(np * 8);
  add(nu * 8); add(nu * 8); add(16 * 8); add(4 * 4); add(dim * nf * 8); add(nf);
  add(nmat * 8);
  for (int i = 0; i < 5; ++i) add(N * 8);
  add(ne * 4); add(16 * 4); add(16 * 8); add(nfn * nf * 8);
  // subdomains, level schedule, record streams, task table, nonlinear list
  add(ne * 4); add((ne + nsd) * 4); add(nsd * 4); add(nsd * 4);  // levels per subdomain <= its elements
  add(ne); add(ne); add(ne * 4);
  add(ne * 8); add(ne * 8); add(ne * 8); add(nsd * 8); add(nsd * 8);
  add(std::max(ncrack, 64LL) * 4);
  // solver workspace of both precisions
  add(ldv * (mres + 1) * 8); for (int i = 0; i < 5; ++i) add(N * 8);
  add(ldv * (mres + 1) * 4); for (int i = 0; i < 5; ++i) add(N * 4);
  add(ne * lus * 8); add(ne * lus * 4); add(std::max(np, 1LL) * 8); add(std::max(np, 1LL) * 4);
  add(nmat * 4); add((long long)std::max(152 * 4 * GM_LD, GS_MAXB_HOST * (2 * GM_MAX + 2)) * 8);
  add(GS_MAXB_HOST * 8);
  add(std::max<long long>(np, 1) * 8); add(std::max<long long>(np, 1) * 8);  // fixed pressures, fluid diagonal
  add((long long)sizeof(GmresState));
  // coarse level (largest layout the options allow: coarse_max = 4096 at most)
  {
    int cA = 0, cnagg = 0, cnc = 0;
    coarse_sizes(ne, (int)dim, o.coarse ? o.coarse_max : 2048, &cA, &cnagg, &cnc);
    const long long nc2 = (long long)cnc * cnc;
    add(cnagg * 4 * 8); add(nu * 8); add(nu * 4); add(nc2 * 8); add((long long)coarse_spare_doubles((int)cnc) * 8); add(nc2 * 4); add(8);
    add(cnc * 8); add(cnc * 8); add(cnc * 4); add(cnc * 4);
  }
  // time-step snapshot
  add(N * 8); add(nfn * nf * 8);
  *bytes = t;
  return HF_OK;
}

}  // extern "C"
