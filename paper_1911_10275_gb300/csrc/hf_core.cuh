// hf_core.cuh - internal data layout and device helpers of the GB300 Newton step.
//
// Layout in HBM (internal element order = Morton order of element centroids):
//   vectors      x[e*ned + a*dim + k] for displacements (element-major, the
//                caller's layout up to the element permutation), then the
//                pressure unknowns at offset nu.
//   J_base       element-block CSR in structure-of-arrays form, element index
//                fastest so that a thread per element reads coalesced:
//                  dg [(c*ned + r)*ne + e]              dense ned x ned block
//                  off[((j*ned + c)*nfr + rr)*ne + e]   facet slot j: rows are
//                  the nfr face rows of e's local facet j, columns the ned
//                  unknowns of the neighbour across it.
//                IIPG flux terms only reach the face nodes of the test side,
//                so these compact blocks hold every structural non-zero.
//   LU factor    array-of-structures, one contiguous record per element so a
//                warp (lane = row) reads coalesced: [Dinv (ned x ned, column
//                major)] then per slot j a (ned cols x nfr rows) block holding
//                L (neighbour eliminated earlier in the same subdomain) or U.
//   nonlinear    small per-facet matrices in the facet's face-node order
//   facet data   (cohesive tangent, pressure mass, lubrication C and D parts).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hfk {

// process-wide count of kernel launches issued by the library (host side)
long long& launch_counter();        // kernels launched by the calling host thread
void add_launches(long long n);     // process-wide total, shared by all threads
long long total_launches();
inline void note_launch() {
  ++launch_counter();
  add_launches(1);
}

constexpr int MAXFN = 6;     // face nodes of a P2 facet (3D)
constexpr int MAXNED = 30;   // unknowns of a P2 tetrahedron
constexpr int MAXNQ = 25;    // nonlinear facet rule size (3D)
constexpr int MAXLQ = 9;     // linear facet rule size (3D)
constexpr int MAXVQ = 8;     // volume rule size (3D)

// face-node order of local facet j (vertices ascending, then edge mid-nodes)
__host__ __device__ constexpr int fn2(int j, int a) {
  return (j == 0) ? (a == 0 ? 1 : a == 1 ? 2 : 4)
       : (j == 1) ? (a == 0 ? 0 : a == 1 ? 2 : 5)
                  : (a == 0 ? 0 : a == 1 ? 1 : 3);
}
__host__ __device__ constexpr int fn3(int j, int a) {
  return (j == 0) ? (a == 0 ? 1 : a == 1 ? 2 : a == 2 ? 3 : a == 3 ? 5 : a == 4 ? 8 : 9)
       : (j == 1) ? (a == 0 ? 0 : a == 1 ? 2 : a == 2 ? 3 : a == 3 ? 6 : a == 4 ? 7 : 9)
       : (j == 2) ? (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 3 : a == 3 ? 4 : a == 4 ? 7 : 8)
                  : (a == 0 ? 0 : a == 1 ? 1 : a == 2 ? 2 : a == 3 ? 4 : a == 4 ? 5 : 6);
}
template <int DIM>
__host__ __device__ constexpr int face_node(int j, int a) { return DIM == 2 ? fn2(j, a) : fn3(j, a); }

// face vertices (p, q) spanned by the mm-th mid-node of local facet j
__host__ __device__ constexpr int midpair3(int j, int mm, int which) {
  return (j < 3) ? (mm == 0 ? (which ? 1 : 0) : mm == 1 ? (which ? 2 : 0) : (which ? 2 : 1))
                 : (mm == 0 ? (which ? 1 : 0) : mm == 1 ? (which ? 2 : 1) : (which ? 2 : 0));
}

// element edge table of the P2 mid-nodes
__host__ __device__ constexpr int edge2(int m, int which) {
  return m == 0 ? (which ? 1 : 0) : m == 1 ? (which ? 2 : 1) : (which ? 0 : 2);
}
__host__ __device__ constexpr int edge3(int m, int which) {
  return m == 0 ? (which ? 1 : 0) : m == 1 ? (which ? 2 : 1) : m == 2 ? (which ? 2 : 0)
       : m == 3 ? (which ? 3 : 0) : m == 4 ? (which ? 3 : 1) : (which ? 3 : 2);
}
template <int DIM>
__host__ __device__ constexpr int edge_v(int m, int which) { return DIM == 2 ? edge2(m, which) : edge3(m, which); }

template <int DIM> struct Shape {
  static constexpr int nv = DIM + 1;                   // vertices / facets
  static constexpr int nen = DIM == 2 ? 6 : 10;        // nodes per element
  static constexpr int ned = nen * DIM;                // unknowns per element
  static constexpr int nfn = DIM == 2 ? 3 : 6;         // nodes per facet
  static constexpr int nfr = nfn * DIM;                // face rows per slot
  static constexpr int lus = ned * ned + nv * ned * nfr;  // LU record size
  static constexpr int nld = 4 * nfn * nfn + 3 * nfn;  // nonlinear facet record
};

// offsets inside the nonlinear facet record
template <int DIM> struct NL {
  static constexpr int F = Shape<DIM>::nfn;
  static constexpr int Tm = 0;            // int T'(w) phi_a phi_b
  static constexpr int Mm = F * F;        // int eta_a phi_b
  static constexpr int Cs = 2 * F * F;    // int (3w^2/12mu grad p.grad eta_a + eta_a/dt) phi_b
  static constexpr int Dm = 3 * F * F;    // int w^3/12mu grad eta_a . grad eta_b
  static constexpr int rc = 4 * F * F;    // int T(w) phi_a
  static constexpr int rp = 4 * F * F + F;      // int p phi_a
  static constexpr int rf = 4 * F * F + 2 * F;  // int (w^3/12mu grad p.grad eta_a + (w - w^n)/dt eta_a)
};

struct Quad {
  int nq_f, nq_l, nq_v;              // nonlinear facet, linear facet, volume
  double f_lam[MAXNQ][3], f_w[MAXNQ];
  double l_lam[MAXLQ][3], l_w[MAXLQ];
  double v_lam[MAXVQ][4], v_w[MAXVQ];
};

struct DevMesh {
  int dim, nen, ned, nfn, nfr, nslot;
  int ne, nf, np, G, nsd;
  long long nu, N;
  // element data (internal order)
  const double* xyz;        // [node*dim + k]
  const int* enode;         // [a*ne + e] global node ids
  double* grad_lam;         // [(i*dim + k)*ne + e]
  double* vol;              // [ne]
  int* nbr;                 // [j*ne + e] neighbour element or -1
  int* slot_face;           // [j*ne + e] facet id or -1
  signed char* slot_side;   // [j*ne + e] 0: e is e_minus, 1: e_plus
  unsigned int* dirmask;    // [ne] Dirichlet rows of e
  unsigned char* nlmask;    // [ne] bit j: cohesive slot, bit 4+j: fluid slot
  unsigned char* lowmask;   // [ne] bit j: slot neighbour eliminated earlier (same subdomain)
  unsigned char* upmask;    // [ne] bit j: slot neighbour eliminated later (same subdomain)
  // facet data (caller facet ids)
  int* fe;                  // [s*nf + f] internal elements (s = 0 minus, 1 plus)
  signed char* fl;          // [s*nf + f] local facet ids
  double* fnormal;          // [k*nf + f]
  double* farea;            // [nf]
  double* fh;               // [nf] min(|e-|,|e+|)/|f|
  double* fsg;              // [(m*dim + k)*nf + f] surface gradient of face barycentric m
  signed char* loc_m;       // [a*nf + f] local node of e_minus at face node a
  signed char* loc_p;       // [a*nf + f] local node of e_plus at face node a
  int* fpdof;               // [a*nf + f] pressure unknown of face node a, or -1
  signed char* crack;       // [nf]
  signed char* alpha;       // [nf]
  signed char* beta;        // [nf]
  double* w_old;            // [a*nf + f] face-node openings at t^n
  double* nl;               // [f*nld + ...] nonlinear facet records
  int* nl_faces;            // list of facets with alpha or beta set
  int n_nl;
  // pressure unknowns
  int* pinc_ptr;            // [np+1] CSR over incident crackable facets
  int* pinc_face;
  signed char* pinc_a;      // face-node index of the pressure node in that facet
  signed char* p_active;    // [np] touches a facet with beta = 1
  double* inj_w;            // [np] injection weights
  double* p_fixval;         // [np] value of an essential (fixed) pressure, NaN where free
  double* sinv_d;           // [np] fluid-only solves: inverse diagonal of the pressure block
  int phase;                // 0 coupled; staggered scheme: 1 mechanics only, 2 fluid only
  // boundary data
  double* ubar;             // [nu] Dirichlet values (0 elsewhere)
  double* fext;             // [nu] Neumann load vector
  // block-Jacobi subdomains
  int* sd_elems;            // [ne] elements of each subdomain, by level
  int* sd_lvl;              // level offsets into sd_elems, per subdomain
  int* sd_lvl_base;         // [nsd] index of the subdomain's first offset in sd_lvl
  int* sd_nlvl;             // [nsd]
  long long* rec_fwd;       // [ne] start of the element's forward segment (L blocks)
  long long* rec_bwd;       // [ne] start of the element's backward segment (U blocks, Dinv)
  unsigned char* sd_task;   // [8 per position in level order]: local id, lower mask, upper mask, -, 4 local nbrs
  long long* sd_fwd;        // [nsd] start of each subdomain's forward stream
  long long* sd_bwd;        // [nsd] start of each subdomain's backward stream
  int* err_flag;            // [0]: a bounded wait in a kernel gave up
  int wait_polls;           // polls of a bounded mbarrier wait before it gives up
  // parameters
  double lam, mu, sigma_c, delta_c, b_stab;
  double mu_f, Q0, delta_f, dt, p_v;
  int cutoff;
  double* scal;             // device scalars: [0] = fluid row scale c^n
};

// ----------------------------------------------------------------------------
// P2 basis on an element in barycentric coordinates
template <int DIM>
__device__ __forceinline__ void p2_vals(const double* lam, double* N) {
#pragma unroll
  for (int i = 0; i < DIM + 1; ++i) N[i] = lam[i] * (2.0 * lam[i] - 1.0);
#pragma unroll
  for (int m = 0; m < Shape<DIM>::nen - DIM - 1; ++m)
    N[DIM + 1 + m] = 4.0 * lam[edge_v<DIM>(m, 0)] * lam[edge_v<DIM>(m, 1)];
}

// gradients: G[a*DIM + k] = sum_i dN_a/dlam_i grad(lam_i)_k ; gl[(i*DIM+k)]
template <int DIM>
__device__ __forceinline__ void p2_grads(const double* lam, const double* gl, double* G) {
#pragma unroll
  for (int i = 0; i < DIM + 1; ++i) {
    double s = 4.0 * lam[i] - 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) G[i * DIM + k] = s * gl[i * DIM + k];
  }
#pragma unroll
  for (int m = 0; m < Shape<DIM>::nen - DIM - 1; ++m) {
    int p = edge_v<DIM>(m, 0), q = edge_v<DIM>(m, 1);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      G[(DIM + 1 + m) * DIM + k] = 4.0 * (lam[q] * gl[p * DIM + k] + lam[p] * gl[q * DIM + k]);
  }
}

// P2 basis on facet j in face barycentrics (face-node order of facet j)
template <int DIM>
__device__ __forceinline__ void face_vals(int j, const double* fl, double* phi) {
#pragma unroll
  for (int m = 0; m < DIM; ++m) phi[m] = fl[m] * (2.0 * fl[m] - 1.0);
  if (DIM == 2) {
    phi[2] = 4.0 * fl[0] * fl[1];
  } else {
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
      phi[3 + mm] = 4.0 * fl[midpair3(j, mm, 0)] * fl[midpair3(j, mm, 1)];
  }
}

// surface gradients of the facet basis; sg[m*DIM + k] = grad_Gamma(face lam_m)
template <int DIM>
__device__ __forceinline__ void face_grads(int j, const double* fl, const double* sg, double* G) {
#pragma unroll
  for (int m = 0; m < DIM; ++m) {
    double s = 4.0 * fl[m] - 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) G[m * DIM + k] = s * sg[m * DIM + k];
  }
  if (DIM == 2) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) G[2 * DIM + k] = 4.0 * (fl[1] * sg[0 * DIM + k] + fl[0] * sg[1 * DIM + k]);
  } else {
#pragma unroll
    for (int mm = 0; mm < 3; ++mm) {
      int p = midpair3(j, mm, 0), q = midpair3(j, mm, 1);
#pragma unroll
      for (int k = 0; k < DIM; ++k)
        G[(3 + mm) * DIM + k] = 4.0 * (fl[q] * sg[p * DIM + k] + fl[p] * sg[q * DIM + k]);
    }
  }
}

// element barycentrics of a facet point given in e_minus's face barycentrics
template <int DIM>
__device__ __forceinline__ void face_to_elem_lam(const DevMesh& m, int f, int side, const double* flam,
                                                 double* lam) {
#pragma unroll
  for (int i = 0; i < DIM + 1; ++i) lam[i] = 0.0;
#pragma unroll
  for (int v = 0; v < DIM; ++v) {
    int loc = side == 0 ? m.loc_m[v * m.nf + f] : m.loc_p[v * m.nf + f];
    lam[loc] = flam[v];
  }
}

// ILU factor layout: per subdomain, a forward stream (the L blocks of its
// lower slots, element after element in level order) followed by a backward
// stream (U blocks of the upper slots then Dinv, element after element in
// reverse level order).  A warp solving the subdomain reads each stream front
// to back.  Blocks hold ned columns x nfr face rows (rows fastest), slots in
// ascending order; Dinv is ned x ned column-major.
__host__ __device__ inline int slots_below(unsigned mask, int j) {
#ifdef __CUDA_ARCH__
  return __popc(mask & ((1u << j) - 1u));
#else
  return __builtin_popcount(mask & ((1u << j) - 1u));
#endif
}
__host__ __device__ inline int nbits(unsigned mask) {
#ifdef __CUDA_ARCH__
  return __popc(mask);
#else
  return __builtin_popcount(mask);
#endif
}

// traction-separation law with the contact penalty for w < 0 and zero
// traction beyond delta_c
__device__ __forceinline__ void tsl(double w, double sc, double dc, double kp, double& T, double& dT) {
  if (w < 0.0) {
    T = sc + kp * w;
    dT = kp;
  } else if (w < dc) {
    T = sc * (1.0 - w / dc);
    dT = -sc / dc;
  } else {
    T = 0.0;
    dT = 0.0;
  }
}

// 16-byte vectors for the Krylov kernels: 4 floats or 2 doubles per load
template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
  __device__ static float dot(const float4& a, const float4& b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
  __device__ static void axpy(float4& y, float a, const float4& x) {
    y.x -= a * x.x; y.y -= a * x.y; y.z -= a * x.z; y.w -= a * x.w;
  }
  __device__ static void fma(float4& y, float a, const float4& x) {
    y.x += a * x.x; y.y += a * x.y; y.z += a * x.z; y.w += a * x.w;
  }
  __device__ static float4 scale(const float4& x, float a) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
  __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  // y += a * b componentwise; the components summed in a fixed order
  __device__ static void madd(float4& y, const float4& a, const float4& b) {
    y.x += a.x * b.x; y.y += a.y * b.y; y.z += a.z * b.z; y.w += a.w * b.w;
  }
  __device__ static float hsum(const float4& a) { return (a.x + a.y) + (a.z + a.w); }
};
template <> struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
  __device__ static double dot(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }
  __device__ static void axpy(double2& y, double a, const double2& x) { y.x -= a * x.x; y.y -= a * x.y; }
  __device__ static void fma(double2& y, double a, const double2& x) { y.x += a * x.x; y.y += a * x.y; }
  __device__ static double2 scale(const double2& x, double a) { return make_double2(a * x.x, a * x.y); }
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static void madd(double2& y, const double2& a, const double2& b) { y.x += a.x * b.x; y.y += a.y * b.y; }
  __device__ static double hsum(const double2& a) { return a.x + a.y; }
};

}  // namespace hfk
