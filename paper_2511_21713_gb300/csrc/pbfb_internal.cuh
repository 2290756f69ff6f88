// Internal declarations of libpbfb: device data of a mesh and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pbfb.h"

namespace pbfb {

void set_error(const char* fmt, ...);
const char* last_error();

#define PB_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      pbfb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? PBFB_ERR_OOM : PBFB_ERR_CUDA;            \
    }                                                                                    \
  } while (0)

#define PB_TRY(call)                 \
  do {                               \
    int s_ = (call);                 \
    if (s_ != PBFB_OK) return s_;    \
  } while (0)

#define PB_LAUNCHED(mesh)                                                                  \
  do {                                                                                     \
    (mesh)->launches++;                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) {                                                               \
      pbfb::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return PBFB_ERR_CUDA;                                                                \
    }                                                                                      \
  } while (0)

// Quadrature points per surface triangle and per tetrahedron.
constexpr int QS = 6;
constexpr int QT = 14;

// Owned device allocation.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    release();
    if (count == 0) return PBFB_OK;
    PB_CUDA(cudaMalloc((void**)&p, count * sizeof(T)));
    n = count;
    return PBFB_OK;
  }
  int upload(const T* h, size_t count, cudaStream_t s) {
    PB_TRY(alloc(count));
    if (count) PB_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    return PBFB_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DBuf() { release(); }
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};

// Special (near-field) triangle pair classes.
enum PairClass { PAIR_IDENTICAL = 0, PAIR_EDGE = 1, PAIR_VERTEX = 2, PAIR_NEAR = 3 };

// Treecode plan of a surface's float32 far field (treecode.cu): quadrature points in tree order,
// target leaves, approximated clusters and their proxies, source tiles grouped into chunks.
struct SurfaceTree {
  bool built = false;
  int nq = 0, nleaf = 0, nclus = 0, nchunk = 0;
  double pairs = 0.0;               // pair evaluations per application (direct + proxy)
  DBuf<int> perm, pos_leaf;         // tree position -> quadrature point; tree position -> leaf
  DBuf<int> leaf_beg, leaf_end, leaf_chunk;  // per leaf: targets [beg, end), chunks [chunk[L], chunk[L+1])
  DBuf<int> chunk_leaf, chunk_tile; // per chunk: its leaf; its tiles [tile[c], tile[c+1])
  DBuf<int2> tiles;                 // per tile: first source record, count (<= 128)
  int npair = 0;                    // runs of leaves in the upward pass
  DBuf<float> clus_box;             // per cluster: lo x, y, z, hi x, y, z (centre-relative)
  DBuf<float> leaf_box;             // per leaf: the same
  DBuf<float4> leaf_prox;           // per leaf: its (p+1)^3 proxies (charge, dipole) from its points
  DBuf<int> pair_clus, pair_leaf, pair_nleaf;  // per run of leaves of one cluster: cluster, first leaf, leaves
  DBuf<int> clus_pair;              // per approximated cluster: its runs [clus_pair[k], clus_pair[k + 1])
  DBuf<float4> up_part;             // per run: its leaves' proxies on the cluster's grid
  DBuf<int> up_arrivals;            // per cluster: runs done in the running upward pass (0 between)
  DBuf<float4> tgt;                 // target positions in tree order
  DBuf<float4> spos, sdl;           // nq points in tree order, then nclus x (p+1)^3 proxies
  DBuf<double> part;                // nchunk x 256 partial sums
};

// A closed surface (Gamma_m or Gamma_s) over shell vertices.
struct Surface {
  int nt = 0;   // triangles
  int nv = 0;   // vertices (unknowns lam)
  int nq = 0;   // quadrature points = QS * nt
  int col0 = 0; // offset of this surface's lam unknowns in the full vector
  std::vector<int> tri_h;   // nt*3 local vertex ids
  std::vector<int> vmap_h;  // nv shell ids (ascending)
  DBuf<int> tri;            // nt*3 local ids
  DBuf<int> vmap;           // nv shell ids
  DBuf<double> qx;          // 3*nq SoA quadrature points (x block, y block, z block)
  DBuf<double> qw;          // nq: w_q |tau|
  DBuf<double> nrm;         // 3*nt SoA unit normals (stored orientation)
  DBuf<double> area;        // nt
  DBuf<float4> qpf;         // nq float (x, y, z, 0) relative to ctr
  double ctr[3] = {0, 0, 0};
  double ff_q = 0.0;            // grid of the float-float coordinates' high parts (a power of 2)
  // test reduction: per vertex list of (tri*3 + a)
  DBuf<int> inc_ptr, inc_idx;
  // special pairs
  int npair = 0;                    // runs of leaves in the upward pass
  DBuf<int> pair_t, pair_s, pair_cls, pair_perm;  // perm: 6 ints per pair (pt[3], ps[3])
  // correction CSR over surface vertices (pattern of all special pairs)
  int cnnz = 0;
  std::vector<int> c_ptr_h, c_col_h;
  DBuf<int> c_ptr, c_col;
  DBuf<int> cg_ptr, cg_idx;     // per slot: pair-local entries p*9 + a*3 + b
  DBuf<int> dg_ptr, dg_idx;     // per vertex: pair-local entries feeding the V diagonal
  DBuf<double> pairV, pairK, pairVfull;  // 9 per pair
  DBuf<double> corrV, corrK;    // per slot: exact-minus-regular corrections
  DBuf<double> mass;            // per slot: P1 mass matrix entries (0 off the mass pattern)
  DBuf<double> diagV;           // per vertex: full single-layer diagonal
  double kappa = -1.0;          // kernel inverse length the corrections were built for
  bool built = false;
  // far-field work buffers
  DBuf<float4> spos, sdl;       // float32 sources
  DBuf<double> s64;             // float64 sources: 7 * nq (x, y, z, s, mx, my, mz)
  DBuf<double> val;             // nsplit * nq target potentials
  DBuf<float4> ffsrc, fftgt;    // float-float sources (4 float4) and targets (2 float4) per point
  int nsplit = 1;
  DBuf<double> mval;            // mutual float32 far field: 2 G partial rows + the sum
  SurfaceTree tree;             // treecode plan of the float32 far field (built on first use)
  // dense single layer (float32, ld x ld): -V^-1 once inverted (bem_dense.cu)
  DBuf<float> vinv;
  int vinv_ld = 0;
  bool vinv_ok = false;
  double vinv_kappa = -1.0;
};

struct KernelClassTimer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double ms = 0.0;
  double count = 0.0;
  double work = 0.0;
};

struct Mesh {
  int dev = 0;
  cudaStream_t stream = 0;
  int nv = 0;
  int64_t nt = 0;
  int n = 0;              // nv + nm + ns
  // geometry
  DBuf<double> xyz;       // 3*nv SoA
  DBuf<int> tets;         // 4*nt SoA (vertex a of tet t at a*nt + t)
  DBuf<double> vol;       // nt
  // sparse part of the coupled operator, CSR over all n rows and n columns
  int snnz = 0;
  std::vector<int> s_ptr_h, s_col_h;
  DBuf<int> s_ptr, s_col;
  DBuf<double> s_val;     // current values (A + J, couplings, BEM near parts)
  DBuf<double> s_base;    // values with J = 0
  DBuf<double> a1;        // per slot: int grad v_i . grad v_j (0 off the stiffness pattern)
  DBuf<int> s_kind, s_ref;  // per slot fill descriptor (see fill kernel)
  DBuf<int> jg_ptr, jg_idx; // per slot: tet-local Jacobian entries (k * nt + t, k in 0..9)
  DBuf<int> ng_ptr, ng_idx; // per vertex: tet-local load entries (a * nt + t)
  int fem_nnz = 0;          // slots in the first nv rows
  // surfaces
  Surface sm, ss;
  // charges
  int nq = 0;
  DBuf<double> qxyz, qz;    // 3*nq SoA, nq
  DBuf<double> coul;        // nm: <sum z/|x-x_k|, psi_i> (no l_B/eps_m)
  bool charges = false;
  // parameters
  double eps_m = 0, eps_s = 0, kappa = 0, T = 0, lB = 0, kT = 0, coef = 0;
  int precision = PBFB_FP64;
  bool params = false;
  // element work buffers
  DBuf<double> tloc;        // 10 * nt Jacobian + 4 * nt load, tet-local
  DBuf<double> wloc;        // omega batch: nomega * 12 * nt
  DBuf<double> red;         // block partial sums
  DBuf<double> scal;        // device scalars: [0,64) omegas, [64, 64+7*64+3) omega dots,
                            // [1000] ion integral, [4000] dot result, [5000, 5502) PCG scalars
  DBuf<double> red2;        // pair-local mass entries during correction builds
  double* pinned = nullptr; // host pinned scratch (4096 doubles)
  // GMRES workspace
  int gm_restart = 0;
  DBuf<double> gV, gw, gz, gr, gdiag, gh, gpart, gtmp;
  bool gw_is_ax = false;    // after gmres: gw holds Acal x for the returned x (its final true residual)
  DBuf<double> gZ;          // flexible GMRES: preconditioned basis (restart x n)
  DBuf<double> gpcg;        // inner PCG vectors (6 x n), then the fixed input and output of the
                            // captured preconditioner graph (n each)
  // non-cooperative block preconditioner captured as a CUDA graph (launch-bound: ~100 small
  // kernels per application); rebuilt when a buffer or setting it was captured with changes
  cudaGraphExec_t pcg_graph = nullptr;
  const void* pcg_graph_key[9] = {};
  int pcg_graph_iters = -1;
  double pcg_graph_nodes = 0;
  bool pcg_graph_off = false;       // capture not possible on this stream (e.g. the legacy stream)
  DBuf<double> gones;       // n ones
  // block preconditioner: FEM block + Robin term on Gamma_s, and its Jacobi diagonal
  int nrobin = 0;
  DBuf<int> robin_slot, robin_ref;  // FEM-row slot (u-u, both on Gamma_s) <- Gamma_s mass slot
  DBuf<double> pval, pdinv;
  DBuf<float> pvalf, pdinvf;        // float32 copies for the mixed precision's cooperative PCG
  DBuf<float> pcgf;                 // its vectors x, r, z, p, q, w (n each; z stays 0 past nv)
  DBuf<double> reac_rec, reac_part; // reaction potentials: Gamma_m point records, chunk partials
  bool pcg_f32 = false;             // the cooperative PCG runs in float32
  int tune_pcg_prec = 0;            // its arithmetic: 0 built-in (float32 in MIXED), 1 float64, 2 float32
  double gs_radius = 1.0;           // sqrt(|Gamma_s| / 4 pi)
  int coop_blocks = 0;              // grid of the cooperative inner PCG (-1: not available)
  int coop_blocks_f32 = 0;          // grid of its float32 form (one block per SM; -1: not available)
  int coop_blocks_pipe = 0;         // blocks of its register-resident pipelined form (one per SM)
  bool no_coop = false;             // never use the grid-barrier PCG (meshes solved concurrently)
  int tune_tpt = 0;                 // float32 far field: targets per thread (0 = heuristic)
  int tune_bps = 0;                 // float32 far field: target blocks per SM for the source split
  int tune_packed = 0;              // float32 far field: 1 = packed f32x2 kernel
  int tune_ff_kernel = 0;           // float-float far field: 1 one target per thread, 2 two (float2),
                                    // 3 mutual pairs (0 = mutual for large surfaces, else 2)
  int tune_ff_bps = 0;              // float-float far field: target blocks per SM (0 = built-in)
  int tune_tree = 0;                // float32 far field: 0 built-in (treecode from TREE_MIN_POINTS
                                    // points), 1 direct sum, 2 treecode
  int spmv_lanes = 0;               // lanes per row of the operator's sparse part (0 = 8; 4, 8, 16)
  int spmv_block = 0;               // threads per block of that SpMV (0 = 256; 128, 256, 512)
  int tune_pcg_bps = 0;             // blocks per SM of the cooperative inner PCG (0 = all that fit)
  int pcg_lanes = 0;                // lanes per row of its sparse product (0 = 8; 4 or 8; 1: the
                                    // sliced-ELL copy, a lane per row)
  bool sell_ok = false;             // sliced-ELL copy of the preconditioner's FEM block built
  int sell_nslice = 0, sell_ne = 0;
  DBuf<int> sell_ptr, sell_col, sell_map;
  DBuf<double> sell_val;
  bool dense_m = false, dense_s = false;  // surface rows of the block preconditioner use V^-1
  DBuf<float> dwork;                // dense single-layer build: W chunk, sweep panels
  DBuf<int> dflag;                  // sweep pivot status
  // Newton workspace
  DBuf<double> xL, xNL, phi, cvec, dvec, du, pvec, tmp, Nvec, bvec, xout, urb;
  std::vector<double> qz_h;  // charges (host copy)
  // statistics
  double launches = 0;
  bool timing = false;
  KernelClassTimer t_nbody, t_nbody64, t_nbodyff, t_spmv, t_elem, t_dense;
  DBuf<float2> ff_tab;      // float-float exp table of the Yukawa kernel
  DBuf<float4> fx_tab;      // float-float exp / sinh / cosh (j/32) tables of the element kernels
  double nbody_flops = 0.0;  // float32 far-field flops issued (18 per Laplace pair, 24 per Yukawa pair)
  double setup_ms[4] = {0, 0, 0, 0};  // mesh_create: validation, surfaces, operator pattern, device set-up
  // FEM over Omega_m and Omega_i (Sec. 2.2, Eq. fembem_matrix): `tets` holds the tets of Omega_i
  // (the nonlinear term and the ion energy), tets_m those of Omega_m (eps_m, no ions).  Gamma_m is
  // an interior interface: its lam_m rows are the identity during the solve, and lam_m is filled
  // afterwards from the Gamma_m boundary integral equation of Sec. 2.3.1
  bool full = false;
  int64_t nt_m = 0;
  DBuf<int> tets_m;                 // 4*nt_m SoA
  DBuf<double> vol_m, a1m;          // Omega_m volumes; per slot: its stiffness (eps_m applied at fill)
  std::vector<double> gm_tri_xyz;   // shell meshes: 9 per Gamma_m triangle (host), for the winding number
  std::vector<double> grid_xyz;     // 3*nv AoS (host), for locating the charges
  std::vector<int> tets_m_h;        // 4*nt_m AoS (host)
  std::vector<int> cell_ptr, cell_tet;  // uniform grid over the Omega_m tets' bounding boxes
  double cell_lo[3] = {0, 0, 0}, cell_h = 1.0;
  int cell_dim[3] = {0, 0, 0};
  DBuf<double> rho;                 // nv: sum_k z_k v_i(x_k) (no 4 pi l_B)
  DBuf<double> pp_val;              // Gamma_m correction pattern: M_m / 2 + corrK_m
  DBuf<double> pp_work;             // post-process vectors: 6 * nm
  ~Mesh() {
    if (pcg_graph) cudaGraphExecDestroy(pcg_graph);
  }
};

// Source splits any far-field launch shape of launch_bem_far can take on nq points: at most
// ceil(nq / 512), and at most one per target block of a 64-blocks-per-SM grid on 152 SMs (the split
// float32 kernels have at least nq / 1024 target blocks, the float-float and float64 ones more).
inline size_t far_splits_max(int64_t nq) {
  const int64_t a = nq / 512 + 2;
  const int64_t b = nq > 0 ? (int64_t)64 * 152 * 1024 / nq + 2 : 2;
  return (size_t)(a < b ? a : b);
}

// ---- whole-solve entry points shared by the C ABI, the batch call and the server
// region: null for a shell mesh (every tet in Omega_i, Gamma_m a boundary), else per tet 0 (Omega_m)
// or 1 (Omega_i) with Gamma_m the interface between them
int mesh_create(const double* xyz, int nv, const int* tets, int64_t nt, const int* gm, int ngm, const int* gs,
                int ngs, cudaStream_t stream, Mesh** out, const int* region = nullptr);
void mesh_destroy(Mesh* m);
int charges_set(Mesh* m, const double* xyz, const double* z, int nq);
int solve_mesh(Mesh* m, double eps_in, double eps_out, double kappa, double T, const pbfb_newton_opts* opts,
               double* x_out_dev, pbfb_result* res);
size_t estimate_bytes(int64_t nv, int64_t nt, int64_t ngm, int64_t ngs, int restart);
// sum_k z_k v_i(x_k) over the Omega_m tets (a mesh with Omega_m); PBFB_ERR_INVALID for a charge
// in none of them
int point_load(Mesh* m, const double* q_xyz, const double* z, int nq, std::vector<double>& rho);
int charges_inside_gamma_m(const Mesh* m, const double* q_xyz, int nq);
int check_charges_inside(const double* tri9, size_t nt, const double* q, int nq, double* w_out);
}  // namespace pbfb
pbfb::Mesh* pbfb_mesh_internal(pbfb_mesh* h);
namespace pbfb {

// ---- quadrature constants (device) and their host initialisation
int init_quadrature();

// ---- fem_kernels.cu
int launch_tet_volumes(Mesh* m, const int* tets, int64_t nt, double* vol);
int launch_stiffness_local(Mesh* m, const int* tets, int64_t nt, const double* vol, double* loc10);
// ff: the tet-local entries are float-float pairs (the mixed precision's sinh-scheme kernels)
int launch_gather(Mesh* m, int nslots, const int* ptr, const int* idx, const double* local,
                  const double* base, double scale, double* out, bool ff = false);
// *ff tells whether loc was written as float-float pairs
int launch_element_nl(Mesh* m, int scheme, const double* u, double coef, double* loc, bool* ff);
int launch_spmv(Mesh* m, const double* x, double* y);
int launch_omega_elements(Mesh* m, int scheme, const double* u, const double* du,
                          const double* omegas_dev, int nomega, double coef, double* loc, bool* ff);
int launch_omega_dots(Mesh* m, int nomega, const double* loc, const double* c, const double* p,
                      double* dots_dev, bool ff);
int launch_ion_energy(Mesh* m, const double* u, double* out_dev);
int launch_fill_operator(Mesh* m);
int launch_csr_spmv(Mesh* m, int nrows, const int* ptr, const int* col, const double* val, const double* x,
                    double* y, bool accumulate);

// ---- bem_kernels.cu
int launch_surface_geometry(Mesh* m, Surface* s);
// test reduction of far-field partials (sums the source splits in place, then reduces per vertex)
int test_reduce(Mesh* m, Surface* s, double* val, int nsplit, double* y, bool accumulate);
int launch_pair_corrections(Mesh* m, Surface* s, double kappa);
int launch_bem_far(Mesh* m, Surface* s, const double* x, const double* lam, double cs, double cd,
                   double kappa, int precision, double* y, bool accumulate);
int launch_bem_far_ff(Mesh* m, Surface* s, const double* x, const double* lam, double cs, double cd,
                      double kappa, double* y, bool accumulate);
int launch_coulomb(Mesh* m);
// reaction potentials of x_L and x_NL at the charges: ur_dev[0, nq) and ur_dev[nq, 2 nq)
int launch_reaction_potentials(Mesh* m, const double* xL, const double* xNL, double* ur_dev);
int bem_apply_noalloc(Mesh* m, int which, int op, const double* x, double* y);

// ---- treecode.cu: hierarchical float32 far field
constexpr int TREE_MIN_POINTS = 65536;  // built-in: treecode for surfaces of at least this many points
bool use_tree(const Mesh* m, const Surface* s);
int build_surface_tree(Mesh* m, Surface* s);
int launch_tree_far(Mesh* m, Surface* s, double kappa, const float4* spos, const float4* sdl, double* val,
                    double* pairs);

// ---- bem_dense.cu: dense float32 single layer of a surface and its inverse
constexpr int DENSE_V_MAX = 40960;  // surface vertices up to which the dense inverse is used
int dense_ld(int n);
size_t dense_bytes(int n);        // the matrix
size_t dense_work_bytes(int n, int nt);  // build scratch (n vertices, nt triangles)
// assemble V (kappa must be the kappa of the surface's corrections); invert: sweep to -V^-1
int build_dense_single_layer(Mesh* m, Surface* s, double kappa, bool invert);
// z = scale * (stored matrix) v over the surface's vertices
int launch_dense_apply(Mesh* m, Surface* s, double scale, const double* v, double* z);
int dense_copy_out(Mesh* m, Surface* s, float scale, float* out, int ld_out);
// launch attributes of the dense kernels, once per device (called by mesh creation)
int init_dense_attributes();

// ---- one application of the block preconditioner (solver.cu), for the autotuner: prepares it at
// the current Jacobian (dense surface blocks if requested) and applies it to v
int block_precond_apply(Mesh* m, const double* v, double* z, int inner_iters, bool dense);

// ---- blas (solver.cu)
int dot(Mesh* m, const double* a, const double* b, int n, double* out_host);
int launch_axpby(Mesh* m, int n, double a, const double* x, double b, const double* y, double* z);
int ensure(DBuf<double>& b, size_t n);

// timing helpers
void timer_begin(Mesh* m, KernelClassTimer& t, cudaEvent_t* ev);
void timer_end(Mesh* m, KernelClassTimer& t, cudaEvent_t ev0, double work);
void timer_flush(KernelClassTimer& t);

}  // namespace pbfb
