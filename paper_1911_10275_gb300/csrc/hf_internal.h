// hf_internal.h - the handle behind the C ABI and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hf.h"
#include "hf_core.cuh"

namespace hfk {

// kernel launchers (hf_assembly.cu)
template <int DIM> void launch_geometry(const DevMesh& m, cudaStream_t st);
template <int DIM>
void launch_build_rows(const DevMesh& m, const Quad& q, const int* elist, int n, double* dg, double* off,
                       cudaStream_t st);
template <int DIM>
void launch_neumann(const DevMesh& m, const Quad& q, const double* ftrac, const signed char* fneu,
                    cudaStream_t st);
template <int DIM> void launch_face_nl(const DevMesh& m, const Quad& q, const double* X, cudaStream_t st);
template <int DIM>
void launch_criterion(const DevMesh& m, const Quad& q, const double* X, double* tmax, int* n_new,
                      cudaStream_t st);
template <int DIM> void launch_openings(const DevMesh& m, const double* X, double* w, cudaStream_t st);
template <int DIM>
void launch_accept(const DevMesh& m, const Quad& q, const double* X, int* n_new, cudaStream_t st);
void launch_fluid_scale(const DevMesh& m, int enabled, double L_ref, cudaStream_t st);

// element-block matrix in structure-of-arrays form
template <typename T> struct EBMat {
  T* dg = nullptr;
  T* off = nullptr;
};

// GMRES workspace of one precision
template <typename T> struct Krylov {
  T* V = nullptr;        // (m+1) basis vectors, stride ldv
  T* w = nullptr;        // Arnoldi work vector
  T* z = nullptr;        // preconditioned vector
  T* u = nullptr;        // combination of the basis
  T* x = nullptr;        // iterate
  T* b = nullptr;        // right-hand side
  T* lu = nullptr;       // ILU records
  T* sinv = nullptr;     // pressure-row Schur diagonal (inverse)
  T* cc = nullptr;       // coarse residual Phi^T r
  T* cy = nullptr;       // coarse solution A0^-1 Phi^T r
  long long ldv = 0;
};

// longest GMRES cycle, and the leading dimension of its Hessenberg matrix
constexpr int GM_MAX = 96;
constexpr int GM_LD = GM_MAX + 1;
// largest grid of the Gram-Schmidt kernels (rows of their partial tables)
constexpr int GS_MAXB_HOST = 256;

// device scalars of the GMRES driver (one record, double precision); the
// host reads back only the leading scalars
struct GmresState {
  double inv_h;          // 1 / h(j+1, j)
  double beta;           // residual norm of the cycle start
  double tol_abs;        // absolute stopping threshold for |g(j+1)|
  double nrm2;           // scratch reduction result
  int done;
  int jlast;
  int iters;
  int skip2;             // 1: the second Gram-Schmidt pass of this step is not needed
  int reorths;           // second Gram-Schmidt passes taken (running count)
  int pad_;
  long long reorth_cols; // basis columns swept by those second passes (running count)
  double g[GM_LD];
  double h2[GM_LD];      // second Gram-Schmidt pass coefficients
  double cs[GM_MAX], sn[GM_MAX];
  double y[GM_MAX];
  double H[GM_LD * GM_MAX];  // Hessenberg, rotated in place (column-major, ld GM_LD)
  double Hr[GM_LD * GM_MAX]; // delayed CGS2: the Hessenberg matrix before rotation
};

// event-timed kernel classes (profiling mode)
enum ProfKind { PK_SPMV = 0, PK_PREC = 1, PK_ORTH = 2, PK_FACTOR = 3, PK_ASSEMBLY = 4, PK_SPMV64 = 5,
                PK_UPDATE = 6, PK_PREC_AUX = 7, PK_COUNT = 8 };
constexpr int PK_REPORTED = 9;  // the classes above plus whole GMRES cycles
constexpr int PROF_EVENTS = 256;
// event pair recorded as graph nodes inside a captured GMRES cycle; j is the
// Arnoldi step it belongs to (-1: once per cycle)
struct GraphEv {
  int kind;
  int j;
  cudaEvent_t a, b;
};

struct Prof {
  bool on = false;
  bool capturing = false;       // events go to the graph being captured
  int cap_j = -1;
  std::vector<GraphEv>* cap_list = nullptr;
  int graph_timing_error = 0;   // CUDA error met reading graph-node events (0: none)
  cudaEvent_t ev[2 * PROF_EVENTS] = {};
  int kind[PROF_EVENTS] = {};
  int n = 0;
  double ms[PK_COUNT] = {};
  long long launches[PK_COUNT] = {};
  // mode 2: whole GMRES cycles timed by an event pair around each launch
  // (graph replay or eager cycle), nothing inside them
  bool cycles = false;
  bool cyc_pending = false;
  cudaEvent_t cyc_a = nullptr, cyc_b = nullptr;
  double cycle_ms = 0.0;
  long long cycle_steps = 0;
};

}  // namespace hfk

struct hf_mesh {
  int dim = 0, nen = 0, ned = 0, nfn = 0, nfr = 0;
  long long ne = 0, nf = 0, nnodes = 0, nu = 0, np = 0, N = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side stream of the preconditioner: the coarse restriction and solve run
  // on it beside the ILU(0) apply (a fork/join that graph capture keeps)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
  bool poisoned = false;
  bool material_set = false, injection_set = false;

  // host bookkeeping
  std::vector<int> ext2int, int2ext;        // element permutation
  std::vector<int> h_fe;                    // [s*nf + f] internal elements
  std::vector<signed char> h_fl, h_crack, h_alpha, h_beta;
  std::vector<int> h_nbr, h_slot_face;      // [j*ne + e]
  std::vector<signed char> h_slot_side;
  std::vector<long long> p_nodes;           // global node of each pressure unknown
  std::vector<int> hp_fpdof;                // [a*nf + f] pressure unknown of face node a
  int nl_cap = 0;                           // capacity of the nonlinear facet list
  int levels_max = 0;                       // deepest level schedule of a subdomain
  std::vector<int> sd_of;                   // subdomain of each internal element
  std::vector<int> sd_always;               // subdomains with a cohesive slot
  std::vector<int> sd_dirty;                // subdomains to refactor once

  // device buffers
  hfk::DevMesh d{};
  hfk::Quad q{};
  struct Alloc {
    void* raw;      // pointer returned by the stream-ordered allocator
    void* base;     // 256-byte aligned start handed out
    size_t bytes;
  };
  std::vector<Alloc> allocs;
  long long bytes_allocated = 0;
  hfk::EBMat<double> J64;
  hfk::EBMat<float> J32;
  bool j32_valid = false;
  double* X = nullptr;         // state [U; P]
  double* R = nullptr;         // residual
  double* D = nullptr;         // Newton increment
  double* tmp64 = nullptr;     // scratch
  double* r64 = nullptr;       // IR residual
  double* fneu_trac = nullptr; // [k*nf + f]
  signed char* fneu = nullptr;
  int* d_elist = nullptr;      // element list scratch
  int* d_sdlist = nullptr;     // subdomain list scratch
  int* d_count = nullptr;      // counters [0]: criterion, [1]: accept, [2..]: reduction counters
  double* d_partial = nullptr; // block partials of reductions
  double* d_part2 = nullptr;   // block partials of the Gram-Schmidt norms (one per CTA)
  int gs_blocks = 0;           // CTAs of the Gram-Schmidt kernels (one per SM)
  long long gs_reorths = 0;    // second Gram-Schmidt passes taken since the workspace was made
  long long gs_reorth_cols = 0; // basis columns those passes swept
  long long gs_cols = 0;       // basis columns swept by first passes: sum over Arnoldi steps of j + 1
  double* d_red = nullptr;     // reduction results
  double* d_wtmp = nullptr;    // facet opening scratch / criterion output
  hfk::GmresState* d_gs = nullptr;
  hfk::Krylov<double> K64;
  hfk::Krylov<float> K32;
  int red_blocks = 0;
  int m_alloc = 0;             // GMRES cycle length the Krylov bases hold

  // parameters
  double E = 0, nu_p = 0, sigma_c = 0, delta_c = 0, b_stab = 10.0;
  double mu_f = 0, Q0 = 0, delta_f = 0, dt = 1.0, p_v = 0, L_ref = 1.0;
  int cutoff = 0;
  double t = 0.0;
  hf_solver_opts opts{};
  int G = 0;                   // subdomain size in use

  // CUDA graphs of one GMRES cycle per precision
  cudaGraphExec_t graph64 = nullptr, graph32 = nullptr;
  std::vector<hfk::GraphEv> gev64, gev32;  // timing events baked into the graphs
  long long graph_kernels64 = 0, graph_kernels32 = 0;  // kernel nodes per captured cycle
  hfk::Prof prof;
  long long n_interior_slots = 0, n_subdomain_slots = 0;

  // coarse level of the preconditioner (hf_coarse.cu)
  int agg_size = 0, nagg = 0, nc = 0;       // elements per aggregate, aggregates, coarse unknowns
  bool coarse_dirty = true;                 // J_base changed since A0 was inverted
  double* agg_geo = nullptr;                // [g*4]: centre (dim), size
  double* rc64 = nullptr;                   // [e*ned + t]: scaled coordinate k of the node of slot t
  float* rc32 = nullptr;
  double* A0a = nullptr;                    // nc x nc: A0, inverted in place
  double* A0b = nullptr;                    // work of the blocked inversion; a spare copy of A0
  double* A0inv64 = nullptr;                // the buffer holding A0^-1
  float* A0inv32 = nullptr;
  double* d_cthr = nullptr;                 // pivot threshold

  // start-of-step snapshot of hf_advance_step (restored when a step is cut)
  double* snap_X = nullptr;
  double* snap_wold = nullptr;
  std::vector<signed char> snap_alpha, snap_beta;
  double snap_t = 0.0;
};

namespace hfk {
// device memory of a handle: stream-ordered on its stream (no device-wide
// synchronisation, so handles on other streams keep running), 256-byte
// aligned, released by dev_free or at hf_mesh_destroy
void* dev_alloc(hf_mesh* h, size_t bytes);
void dev_free(hf_mesh* h, void* p);
// coarse level (hf_coarse.cu)
void coarse_sizes(long long ne, int dim, int coarse_max, int* A, int* nagg, int* nc);
hf_status coarse_layout(hf_mesh* h);
hf_status coarse_refactor(hf_mesh* h);
size_t coarse_spare_doubles(int nc);
hf_status coarse_rebuild_copy(hf_mesh* h, double* A0_host, double* inv_host, double* geo_host);
template <typename T, int DIM>
void coarse_pre(hf_mesh* h, const Krylov<T>& K, const T* rin, const int* skip, cudaStream_t st);
template <typename T, int DIM> void coarse_post(hf_mesh* h, const Krylov<T>& K, T* z, const int* skip);
// solver side (hf_solve.cu)
hf_status solver_alloc(hf_mesh* h);
hf_status krylov_basis_alloc(hf_mesh* h, int m);
void convert_j32(hf_mesh* h);
void factor_subdomains(hf_mesh* h, const std::vector<int>& sds);
hf_status residual(hf_mesh* h, const double* X, double* R);
hf_status apply_jacobian(hf_mesh* h, const double* x, double* y);
hf_status linear_solve(hf_mesh* h, const double* b, double* x, hf_newton_report* rep);
hf_status newton_update(hf_mesh* h, const double* Dx, double out[4]);
void launch_neg_part(hf_mesh* h, const double* R, double* b, int keep_u, int keep_p);
void launch_diag_d(hf_mesh* h);
void launch_wait_selftest(hf_mesh* h);
double device_norm2(hf_mesh* h, const double* v, long long n);
hf_status set_error(hf_mesh* h, hf_status s, const std::string& msg);
hf_status check_cuda(hf_mesh* h, cudaError_t e, const char* where);
// profiling: event pair around a kernel class; flush accumulates elapsed times
void prof_begin(hf_mesh* h, int kind);
void prof_end(hf_mesh* h);
void prof_flush(hf_mesh* h);
}  // namespace hfk
