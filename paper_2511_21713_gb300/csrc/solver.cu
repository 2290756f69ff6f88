// Coupled operator, GMRES, Newton-Raphson with the optimal relaxation factor, energy,
// and the C ABI (include/pbfb.h).
//
// Newton (Sec. 2.4.2, Eqs. NR_main, Ec_NL_NR, Norma_Newton-Raphson): with Phi = x_L + x_NL,
//   d = b - Acal(0) Phi - [N(u);0;0],  Acal(J(u)) Delta = d,  x_NL += omega Delta,
//   e = omega ||Delta||_2, stop when e < Tol_NL; T3 nonlinearity in the first iteration.
// Relaxation factor (Sec. 2.5, Eq. fd=0, Appendix A): Newton's method on
//   f_d(omega) = -((p + r').r) / ((p + r').p) - omega, p = -Acal(0) Delta,
// accepted when 0 < omega <= omega_max and ||d(omega)|| < ||d(0)|| (the global convergence
// condition of Sec. 2.5.2); otherwise a batched scan of g_d = d . d' over omega_max j / 16
// followed by bisection of its first sign change.  L_e skip rule and the adjustable GMRES
// tolerance follow Appendix B.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "pbfb_internal.cuh"
#include "warp_sum.cuh"

namespace pbfb {

const char* last_error();

namespace {

// e^2/(4 pi eps0) in kcal mol^-1 Angstrom and the Boltzmann constant in kcal mol^-1 K^-1.
constexpr double kCoulomb = 332.0637;
constexpr double kBoltzmann = 0.0019872043;
constexpr int DOT_B = 152;
constexpr int DOT_T = 256;

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_dot_partial(int n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ part) {
  double acc = 0.0;
  for (int i = blockIdx.x * DOT_T + threadIdx.x; i < n; i += gridDim.x * DOT_T) acc += a[i] * b[i];
  __shared__ double sh[DOT_T / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < DOT_T / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// one warp: *out = sum of the nb partials (fixed order)
__global__ void k_sum_to(const double* __restrict__ part, int nb, double* __restrict__ out) {
  const double s = warp_strided_sum(part, nb, 1);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpby(int n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ z) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

__global__ void k_mul(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ z) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a[i] * b[i];
}

__global__ void k_scale_by(int n, const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / sqrt(*s);
}

// h[j] partials: for basis vectors j0..j0+7 (< k), sum over a row range of V[j] . w
constexpr int MD_T = 256;
__global__ void __launch_bounds__(MD_T) k_multidot(int n, int k, const double* __restrict__ V,
                                                   const double* __restrict__ w, double* __restrict__ part) {
  int j0 = blockIdx.y * 8;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * MD_T + threadIdx.x; i < n; i += gridDim.x * MD_T) {
    double wi = w[i];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (j0 + jj < k) acc[jj] += V[(int64_t)(j0 + jj) * n + i] * wi;
  }
  __shared__ double sh[MD_T / 32][8];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    double x = acc[jj];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][jj] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8 && j0 + (int)threadIdx.x < k) {
    double x = 0.0;
    for (int q = 0; q < MD_T / 32; ++q) x += sh[q][threadIdx.x];
    part[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = x;
  }
}

// one warp per j: h[j] = sum of its nb partials (fixed order)
__global__ void k_multidot_sum(const double* __restrict__ part, int nb, int k, double* __restrict__ h) {
  const int j = blockIdx.x;
  if (j >= k) return;
  const double s = warp_strided_sum(part + (int64_t)j * nb, nb, 1);
  if (threadIdx.x == 0) h[j] = s;
}

// w -= sum_j V[j] h[j]; optional partial sums of ||w||^2 after the update
__global__ void __launch_bounds__(MD_T) k_multiaxpy(int n, int k, const double* __restrict__ V,
                                                    const double* __restrict__ h, double* __restrict__ w,
                                                    double* __restrict__ npart) {
  double nrm = 0.0;
  for (int i = blockIdx.x * MD_T + threadIdx.x; i < n; i += gridDim.x * MD_T) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += V[(int64_t)j * n + i] * h[j];
    double v = w[i] - s;
    w[i] = v;
    nrm += v * v;
  }
  if (!npart) return;
  __shared__ double sh[MD_T / 32];
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < MD_T / 32; ++q) s += sh[q];
    npart[blockIdx.x] = s;
  }
}

// x += dinv .* (sum_j V[j] y[j])
__global__ void k_update_solution(int n, int k, const double* __restrict__ V, const double* __restrict__ y,
                                  const double* __restrict__ dinv, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s += V[(int64_t)j * n + i] * y[j];
  x[i] += dinv[i] * s;
}

// Jacobi preconditioner: 1 / diag(Acal(J)).  FEM rows from the sparse part; surface rows
// from the full single-layer diagonals (-V_L on Gamma_m, +V_Y on Gamma_s).
__global__ void k_jacobi(int nv, int nm, int ns, const int* __restrict__ ptr, const int* __restrict__ col,
                         const double* __restrict__ val, const double* __restrict__ dVm,
                         const double* __restrict__ dVs, double* __restrict__ dinv) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nv + nm + ns) return;
  double d;
  if (r < nv) {
    d = 0.0;
    for (int k = ptr[r]; k < ptr[r + 1]; ++k)
      if (col[k] == r) d = val[k];
  } else if (r < nv + nm) {
    d = dVm ? -dVm[r - nv] : 1.0;  // no dVm: identity rows of an interior Gamma_m
  } else {
    d = dVs[r - nv - nm];
  }
  dinv[r] = 1.0 / d;
}

// ---- Jacobi-PCG on the FEM block (rows < nv of the sparse part; the search direction
// is kept zero on the surface unknowns so the coupling columns contribute nothing).
constexpr int PCG_T = 256;

__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double sh[PCG_T / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < PCG_T / 32; ++w) s += sh[w];
    *out = s;
  }
  __syncthreads();  // sh is reused by the next call
}

// x = 0, r = b, z = dinv r, p = z, partial r.z
__global__ void __launch_bounds__(PCG_T) k_pcg_init(int nv, const double* __restrict__ b,
                                                     const double* __restrict__ dinv, double* __restrict__ x,
                                                     double* __restrict__ r, double* __restrict__ z,
                                                     double* __restrict__ p, double* __restrict__ part) {
  double acc = 0.0;
  for (int i = blockIdx.x * PCG_T + threadIdx.x; i < nv; i += gridDim.x * PCG_T) {
    double bi = b[i], zi = dinv[i] * bi;
    x[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    acc += bi * zi;
  }
  block_sum_store(acc, part + blockIdx.x);
}

// q = (A + J) p on the FEM rows (8 lanes per row), partial p.q
__global__ void __launch_bounds__(PCG_T) k_pcg_spmv(int nv, const int* __restrict__ ptr,
                                                     const int* __restrict__ col, const double* __restrict__ val,
                                                     const double* __restrict__ p, double* __restrict__ q,
                                                     double* __restrict__ part) {
  // warp-uniform trip count: every lane of a warp executes every shuffle (4 rows per warp pass)
  const int lane = threadIdx.x & 7;
  const int warp = (blockIdx.x * PCG_T + threadIdx.x) >> 5, nwarp = (gridDim.x * PCG_T) >> 5;
  double acc = 0.0;
  for (int base = 4 * warp; base < nv; base += 4 * nwarp) {
    const int row = base + ((threadIdx.x & 31) >> 3);
    const bool valid = row < nv;
    double s = 0.0;
    if (valid)
      for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 8) s += val[k] * p[col[k]];
    s += __shfl_down_sync(0xffffffffu, s, 4, 8);
    s += __shfl_down_sync(0xffffffffu, s, 2, 8);
    s += __shfl_down_sync(0xffffffffu, s, 1, 8);
    if (lane == 0 && valid) {
      q[row] = s;
      acc += p[row] * s;
    }
  }
  block_sum_store(acc, part + blockIdx.x);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = dinv r; partial r.z
__global__ void __launch_bounds__(PCG_T) k_pcg_update(int nv, const double* __restrict__ rz,
                                                       const double* __restrict__ pq, double* __restrict__ x,
                                                       double* __restrict__ r, const double* __restrict__ p,
                                                       const double* __restrict__ q, const double* __restrict__ dinv,
                                                       double* __restrict__ z, double* __restrict__ part) {
  const double alpha = (*pq != 0.0) ? (*rz / *pq) : 0.0;
  double acc = 0.0;
  for (int i = blockIdx.x * PCG_T + threadIdx.x; i < nv; i += gridDim.x * PCG_T) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    double zi = dinv[i] * ri;
    z[i] = zi;
    acc += ri * zi;
  }
  block_sum_store(acc, part + blockIdx.x);
}

// beta = rz_new / rz_old; p = z + beta p
__global__ void k_pcg_direction(int nv, const double* __restrict__ rz_old, const double* __restrict__ rz_new,
                                const double* __restrict__ z, double* __restrict__ p) {
  const double beta = (*rz_old != 0.0) ? (*rz_new / *rz_old) : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) p[i] = z[i] + beta * p[i];
}

__global__ void k_to_f32(int n, const double* __restrict__ a, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)a[i];
}

// preconditioner FEM block: pval += c M_s on the Gamma_s u-u slots
__global__ void k_add_robin(int nr, const int* __restrict__ slot, const int* __restrict__ ref,
                            const double* __restrict__ mass, double c, double* __restrict__ pval) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) pval[slot[k]] += c * mass[ref[k]];
}

// Jacobi diagonal of the preconditioner's FEM block
__global__ void k_diag_inv(int nv, const int* __restrict__ ptr, const int* __restrict__ col,
                           const double* __restrict__ val, double* __restrict__ dinv) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nv) return;
  double d = 0.0;
  for (int k = ptr[r]; k < ptr[r + 1]; ++k)
    if (col[k] == r) d = val[k];
  dinv[r] = 1.0 / d;
}

// One thread's part of a step's scalars: alpha and beta from gamma = (r, z) and delta = (z, w) and
// the recurrence state st = {gamma_old, alpha_old, gamma_0} (st[3], st[4] receive alpha and beta).
// f32_rules adds the float32 forms' stops: r.z at 1e-12 of its first value, or a non-positive or
// huge alpha.  A zero r.z (e.g. a right-hand side that vanishes on the FEM rows) gives
// alpha = beta = 0: nothing left to do.  Returns 1 to stop before this step's update.
__device__ __forceinline__ int cg_scalars_lane0(double gamma, double delta, int it, bool f32_rules, double* st) {
  if (it == 0) {
    st[0] = 1.0;
    st[1] = 1.0;
    st[2] = gamma;
  }
  const double gamma_old = st[0], alpha_old = st[1];
  double beta = 0.0, alpha = 0.0;
  if (gamma != 0.0) {
    if (it == 0 || gamma_old == 0.0 || alpha_old == 0.0) {
      alpha = delta != 0.0 ? gamma / delta : 0.0;
    } else {
      beta = gamma / gamma_old;
      const double den = delta - beta * gamma / alpha_old;
      alpha = den != 0.0 ? gamma / den : 0.0;
    }
  }
  int s = 0;
  if (f32_rules && (!(gamma > 1e-12 * st[2]) || !(alpha > 0.0 && alpha < 3e38 && fabs(beta) < 3e38))) s = 1;
  st[0] = gamma;
  st[1] = alpha;
  st[3] = alpha;
  st[4] = beta;
  return s;
}

// The scalars of a Chronopoulos-Gear step from the two grid sums: warp 0 of every block reads the
// per-block partials lane-strided (lane l sums entries l, l + 32, ... in that order), then a
// butterfly over the 32 lanes, so every block obtains the same two sums; lane 0 alone takes the
// divisions and the stop rules (cg_scalars_lane0), and the block reads alpha and beta from shared
// memory (GB300's float64 rate makes two divisions in every thread of the grid the larger part of
// a step).  The recurrence state lives in shared memory, so every block evolves it identically.
// Returns true when the iteration is to stop before this step's update.
__device__ __forceinline__ bool cg_step_scalars(const double* pa, const double* pb, int nb, int it, bool f32_rules,
                                                double* alpha_out, double* beta_out) {
  __shared__ double st[5];  // gamma_old, alpha_old, gamma_0, alpha, beta
  __shared__ int stop;
  if (threadIdx.x < 32) {
    // lane l adds entries l, l + 32, ... in that order, loaded 8 at a time (independent loads)
    double sa = 0.0, sb = 0.0;
    for (int k0 = threadIdx.x; k0 < nb; k0 += 32 * 8) {
      double va[8], vb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 32 * u;
        va[u] = k < nb ? pa[k] : 0.0;
        vb[u] = k < nb ? pb[k] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (k0 + 32 * u < nb) {
          sa += va[u];
          sb += vb[u];
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) stop = cg_scalars_lane0(sa, sb, it, f32_rules, st);
  }
  __syncthreads();
  *alpha_out = st[3];
  *beta_out = st[4];
  const bool s = stop != 0;
  __syncthreads();
  return s;
}

// The whole inner PCG in one cooperative launch (all blocks resident; grid-wide barriers between
// the dependent phases).  Every block sums the per-block partials itself in the same fixed order,
// so all blocks see identical scalars and the result is deterministic.  part: 2 * gridDim.x.
// Chronopoulos-Gear form of preconditioned CG (one fused reduction per step): with w = A z,
// gamma = r.z, delta = z.w: beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
// p = z + beta p, q = w + beta q (= A p), x += alpha p, r -= alpha q, z = M r.  Same iterates as
// standard PCG in exact arithmetic, two grid-wide barriers per step instead of three.
template <int L>
__global__ void __launch_bounds__(PCG_T) k_pcg_coop(int nv, int iters, const int* __restrict__ ptr,
                                                     const int* __restrict__ col, const double* __restrict__ val,
                                                     const double* __restrict__ b, const double* __restrict__ dinv,
                                                     double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ z, double* __restrict__ p,
                                                     double* __restrict__ q, double* __restrict__ w,
                                                     double* __restrict__ part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int nb = gridDim.x;
  double* part_g = part;
  double* part_d = part + nb;
  const int tid = blockIdx.x * PCG_T + threadIdx.x, stride = nb * PCG_T;
  const int lane = threadIdx.x & (L - 1);
  constexpr int RW = 32 / L;  // rows per warp pass
  for (int i = tid; i < nv; i += stride) {
    double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    z[i] = dinv[i] * bi;
    p[i] = 0.0;
    q[i] = 0.0;
  }
  grid.sync();
  for (int it = 0; it < iters; ++it) {
    // w = A z; partial r.z and z.w
    double ag = 0.0, ad = 0.0;
    // warp-uniform trip count: every lane of a warp executes every shuffle (RW rows per warp pass)
    for (int base = RW * (tid >> 5); base < nv; base += RW * (stride >> 5)) {
      const int row = base + (threadIdx.x & 31) / L;
      const bool valid = row < nv;
      double sacc = 0.0;
      if (valid)
        for (int k = ptr[row] + lane; k < ptr[row + 1]; k += L) sacc += val[k] * z[col[k]];
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o, L);
      if (lane == 0 && valid) {
        w[row] = sacc;
        double zr = z[row];
        ag += r[row] * zr;
        ad += zr * sacc;
      }
    }
    block_sum_store(ag, part_g + blockIdx.x);
    block_sum_store(ad, part_d + blockIdx.x);
    grid.sync();
    double alpha, beta;
    cg_step_scalars(part_g, part_d, nb, it, false, &alpha, &beta);
    for (int i = tid; i < nv; i += stride) {
      double pi = z[i] + beta * p[i];
      double qi = w[i] + beta * q[i];
      p[i] = pi;
      q[i] = qi;
      x[i] += alpha * pi;
      double ri = r[i] - alpha * qi;
      r[i] = ri;
      z[i] = dinv[i] * ri;
    }
    grid.sync();
  }
}

// The same iteration in float32 (the mixed precision's preconditioner: flexible GMRES needs no
// exact inner solve, and GB300's float64 rate is 1/64 of its float32 rate): float32 matrix and
// vectors, per-thread float32 dot partials, block and grid sums in float64, scalars in float64.
// One block of PCG_F32_T threads per SM (at most 64 registers a thread), so that a grid barrier
// waits on 152 blocks while 32 warps per SM hide the gathers' latency; the row products issue
// four gathers before their FMAs.  b and the result x_out are float64.  The iteration stops
// early at float32 rounding or before a non-finite or non-positive step: x keeps its last iterate.
constexpr int PCG_F32_T = 1024;

template <int L>
__global__ void __launch_bounds__(PCG_F32_T, 1)
    k_pcg_coop_f32(int nv, int iters, const int* __restrict__ ptr, const int* __restrict__ col,
                   const float* __restrict__ val, const double* __restrict__ b, const float* __restrict__ dinv,
                   double* __restrict__ x_out, float* __restrict__ x, float* __restrict__ r, float* __restrict__ z,
                   float* __restrict__ p, float* __restrict__ q, float* __restrict__ w, double* __restrict__ part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[2][PCG_F32_T / 32];
  const int nb = gridDim.x;
  double* part_g = part;
  double* part_d = part + nb;
  const int tid = blockIdx.x * PCG_F32_T + threadIdx.x, stride = nb * PCG_F32_T;
  const int lane = threadIdx.x & (L - 1);
  constexpr int RW = 32 / L;
  for (int i = tid; i < nv; i += stride) {
    const float bi = (float)b[i];
    x[i] = 0.f;
    r[i] = bi;
    z[i] = dinv[i] * bi;
    p[i] = 0.f;
    q[i] = 0.f;
  }
  grid.sync();
  for (int it = 0; it < iters; ++it) {
    float ag = 0.f, ad = 0.f;
    for (int base = RW * (tid >> 5); base < nv; base += RW * (stride >> 5)) {
      const int row = base + (threadIdx.x & 31) / L;
      const bool valid = row < nv;
      float sacc = 0.f;
      if (valid) {
        int k = ptr[row] + lane;
        const int e = ptr[row + 1];
        for (; k + 3 * L < e; k += 4 * L) {
          const int c0 = col[k], c1 = col[k + L], c2 = col[k + 2 * L], c3 = col[k + 3 * L];
          const float v0 = val[k], v1 = val[k + L], v2 = val[k + 2 * L], v3 = val[k + 3 * L];
          const float z0 = z[c0], z1 = z[c1], z2 = z[c2], z3 = z[c3];
          sacc = fmaf(v0, z0, sacc);
          sacc = fmaf(v1, z1, sacc);
          sacc = fmaf(v2, z2, sacc);
          sacc = fmaf(v3, z3, sacc);
        }
        for (; k < e; k += L) sacc = fmaf(val[k], z[col[k]], sacc);
      }
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o, L);
      if (lane == 0 && valid) {
        w[row] = sacc;
        const float zr = z[row];
        ag = fmaf(r[row], zr, ag);
        ad = fmaf(zr, sacc, ad);
      }
    }
    // block sums: warp shuffles in float32, the warps' values added in float64 in warp order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ag += __shfl_down_sync(0xffffffffu, ag, o);
      ad += __shfl_down_sync(0xffffffffu, ad, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = ag;
      red[1][threadIdx.x >> 5] = ad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sg = 0.0, sd = 0.0;
      for (int k = 0; k < PCG_F32_T / 32; ++k) {
        sg += red[0][k];
        sd += red[1][k];
      }
      part_g[blockIdx.x] = sg;
      part_d[blockIdx.x] = sd;
    }
    grid.sync();
    // the same decision in every block (identical sums): stop once r.z has fallen to float32
    // rounding (1e-12 of its first value: the residual down by about 1e6), and before a
    // non-finite or non-positive step (rounding past convergence)
    double alpha, beta;
    if (cg_step_scalars(part_g, part_d, nb, it, true, &alpha, &beta)) break;
    const float a = (float)alpha, bt = (float)beta;
    for (int i = tid; i < nv; i += stride) {
      const float pi = fmaf(bt, p[i], z[i]);
      const float qi = fmaf(bt, q[i], w[i]);
      p[i] = pi;
      q[i] = qi;
      x[i] = fmaf(a, pi, x[i]);
      const float ri = fmaf(-a, qi, r[i]);
      r[i] = ri;
      z[i] = dinv[i] * ri;
    }
    grid.sync();
  }
  for (int i = tid; i < nv; i += stride) x_out[i] = (double)x[i];
}

// The float32 form with its state resident in registers, for meshes of at most PCG_RES_ROWS rows
// per SM, in the pipelined form of Ghysels and Vanroose (2014): with u = M r, w = A u, m = M w and
// n = A m, every vector is updated by its own recurrence (z = n + beta z, q = m + beta q,
// s = w + beta s, p = u + beta p; x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z), so that
// the dot products of the next step, (r, u) and (w, u), are taken right after an update and pass
// the same grid barrier as m: one barrier per step instead of two.  Same iterates as the
// Chronopoulos-Gear form in exact arithmetic.  Warp 0 of a block owns no rows: while warps 1..31
// gather m for their row products, it adds the block partials of the step's two dots and takes
// the scalars (cg_step_scalars' arithmetic), so the float64 sums and divisions stay off the
// critical path.  A thread owns one row for the whole solve: its row of the FEM block (at most
// PCG_RES_CAP entries in registers; longer rows read the rest each step; the coupling columns past
// nv are dropped) and its x, r, u, w, m, z, q, s, p and diagonal.  Blocks of 1 + 15 warps, one
// per SM (4 warps per SM sub-partition: up to 128 registers a thread).  m and the block partials are double-buffered by step parity: a step reads one buffer
// while it writes the other, and the barrier separates the two uses.
// one row's product with a vector in global memory: the register-held entries, then the rest
__device__ __forceinline__ float pipe_row_product(const int (&cidx)[16], const float (&cval)[16], int k_more,
                                                  int k_end, const int* __restrict__ col,
                                                  const float* __restrict__ val, int nv,
                                                  const float* __restrict__ v) {
  float g[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) g[t] = v[cidx[t]];
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < 16; ++t) acc = fmaf(cval[t], g[t], acc);
  for (int k = k_more; k < k_end; ++k) {
    const int c = col[k];
    if (c < nv) acc = fmaf(val[k], v[c], acc);
  }
  return acc;
}

constexpr int PCG_RES_CAP = 16;  // (pipe_row_product's register entries)
constexpr int PCG_RES_ROWS = 480;
constexpr int PCG_PIPE_T = 32 + PCG_RES_ROWS;

__global__ void __launch_bounds__(PCG_PIPE_T, 1)
    k_pcg_pipe_f32(int nv, int iters, const int* __restrict__ ptr, const int* __restrict__ col,
                   const float* __restrict__ val, const double* __restrict__ b, const float* __restrict__ dinv,
                   double* __restrict__ x_out, float* __restrict__ mbuf, float* __restrict__ ubuf,
                   double* __restrict__ part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ float red[2][PCG_PIPE_T / 32];
  __shared__ double st[5];
  __shared__ int stop;
  const int nb = gridDim.x;
  const int warp = threadIdx.x >> 5;
  const int row = blockIdx.x * PCG_RES_ROWS + (int)threadIdx.x - 32;
  const bool valid = warp > 0 && row < nv;
  const bool owner = valid;
  int cidx[PCG_RES_CAP];
  float cval[PCG_RES_CAP];
  int k_more = 0, k_end = 0;  // entries past the register capacity: [k_more, k_end)
  float x = 0.f, r = 0.f, u = 0.f, w = 0.f, m = 0.f, z = 0.f, q = 0.f, sv = 0.f, p = 0.f, di = 0.f;
  if (valid) {
    const int k0 = ptr[row], e = ptr[row + 1];
#pragma unroll
    for (int t = 0; t < PCG_RES_CAP; ++t) {
      const int k = k0 + t;
      const int c = k < e ? col[k] : nv;
      cidx[t] = c < nv ? c : row;
      cval[t] = c < nv ? val[k] : 0.f;
    }
    k_more = k0 + PCG_RES_CAP;
    k_end = e;
  } else {
#pragma unroll
    for (int t = 0; t < PCG_RES_CAP; ++t) {
      cidx[t] = 0;
      cval[t] = 0.f;
    }
  }
  // block sums of (r, u) and (w, u) into the partials of buffer `buf` (warp sums in float32, the
  // warps' values added in float64 in warp order by warp 0)
  auto block_dots = [&](int buf) {
    float ag = owner ? r * u : 0.f, ad = owner ? w * u : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ag += __shfl_down_sync(0xffffffffu, ag, o);
      ad += __shfl_down_sync(0xffffffffu, ad, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][warp] = ag;
      red[1][warp] = ad;
    }
    __syncthreads();
    if (warp == 0) {
      const bool in = threadIdx.x < PCG_PIPE_T / 32;
      double sg = in ? red[0][threadIdx.x] : 0.0, sd = in ? red[1][threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
      }
      if (threadIdx.x == 0) {
        part[(size_t)buf * 2 * nb + blockIdx.x] = sg;
        part[(size_t)buf * 2 * nb + nb + blockIdx.x] = sd;
      }
    }
  };
  // warp 0: the grid sums of buffer `buf` and the scalars of step it into st[3], st[4]
  auto scalars = [&](int buf, int it) {
    const double* pa = part + (size_t)buf * 2 * nb;
    const double* pb = pa + nb;
    double sa = 0.0, sb = 0.0;
    for (int k0 = threadIdx.x; k0 < nb; k0 += 32 * 8) {
      double va[8], vb[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int k = k0 + 32 * t;
        va[t] = k < nb ? pa[k] : 0.0;
        vb[t] = k < nb ? pb[k] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (k0 + 32 * t < nb) {
          sa += va[t];
          sb += vb[t];
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) stop = cg_scalars_lane0(sa, sb, it, true, st);
  };
  // x = 0, r = b, u = M r; w = A u; m = M w
  if (owner) {
    di = dinv[row];
    r = (float)b[row];
    u = di * r;
    ubuf[row] = u;
  }
  grid.sync();
  {
    const float wu = valid ? pipe_row_product(cidx, cval, k_more, k_end, col, val, nv, ubuf) : 0.f;
    if (owner) {
      w = wu;
      m = di * w;
      mbuf[row] = m;
    }
  }
  block_dots(0);
  grid.sync();
  for (int it = 0; it < iters; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    float n = 0.f;
    if (warp == 0)
      scalars(cur, it);
    else
      n = valid ? pipe_row_product(cidx, cval, k_more, k_end, col, val, nv, mbuf + (size_t)cur * nv) : 0.f;
    __syncthreads();
    if (stop) break;  // identical sums in every block: the same decision everywhere
    if (owner) {
      const float a = (float)st[3], bt = (float)st[4];
      z = fmaf(bt, z, n);
      q = fmaf(bt, q, m);
      sv = fmaf(bt, sv, w);
      p = fmaf(bt, p, u);
      x = fmaf(a, p, x);
      r = fmaf(-a, sv, r);
      u = fmaf(-a, q, u);
      w = fmaf(-a, z, w);
      m = di * w;
      mbuf[(size_t)nxt * nv + row] = m;
    }
    if (it + 1 < iters) {
      block_dots(nxt);
      grid.sync();
    }
  }
  if (owner) x_out[row] = (double)x;
}

// The same iteration with the FEM block in sliced ELL form (slices of 32 consecutive rows, each
// stored column by column at the slice's largest row length, padding entries with value 0): a
// warp takes a slice, a lane a row, so the value and column loads are coalesced and the products
// of a row are independent loads rather than a chain.  Sums in a row run in stored column order.
__global__ void __launch_bounds__(PCG_T) k_pcg_coop_sell(int nv, int nslice, int iters, const int* __restrict__ sptr,
                                                          const int* __restrict__ scol,
                                                          const double* __restrict__ sval,
                                                          const double* __restrict__ b, const double* __restrict__ dinv,
                                                          double* __restrict__ x, double* __restrict__ r,
                                                          double* __restrict__ z, double* __restrict__ p,
                                                          double* __restrict__ q, double* __restrict__ w,
                                                          double* __restrict__ part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int nb = gridDim.x;
  double* part_g = part;
  double* part_d = part + nb;
  const int tid = blockIdx.x * PCG_T + threadIdx.x, stride = nb * PCG_T;
  const int lane = threadIdx.x & 31, gw = tid >> 5, nw = stride >> 5;
  for (int i = tid; i < nv; i += stride) {
    double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    z[i] = dinv[i] * bi;
    p[i] = 0.0;
    q[i] = 0.0;
  }
  grid.sync();
  for (int it = 0; it < iters; ++it) {
    double ag = 0.0, ad = 0.0;
    for (int sl = gw; sl < nslice; sl += nw) {
      const int e0 = sptr[sl], wd = (sptr[sl + 1] - e0) >> 5;
      const int* cp = scol + e0 + lane;
      const double* vp = sval + e0 + lane;
      double sacc = 0.0;
#pragma unroll 4
      for (int j = 0; j < wd; ++j) sacc += vp[32 * j] * z[cp[32 * j]];
      const int row = 32 * sl + lane;
      if (row < nv) {
        w[row] = sacc;
        const double zr = z[row];
        ag += r[row] * zr;
        ad += zr * sacc;
      }
    }
    block_sum_store(ag, part_g + blockIdx.x);
    block_sum_store(ad, part_d + blockIdx.x);
    grid.sync();
    double alpha, beta;
    cg_step_scalars(part_g, part_d, nb, it, false, &alpha, &beta);
    for (int i = tid; i < nv; i += stride) {
      double pi = z[i] + beta * p[i];
      double qi = w[i] + beta * q[i];
      p[i] = pi;
      q[i] = qi;
      x[i] += alpha * pi;
      double ri = r[i] - alpha * qi;
      r[i] = ri;
      z[i] = dinv[i] * ri;
    }
    grid.sync();
  }
}

// sliced-ELL values of the preconditioner's FEM block from its CSR values (padding: 0)
__global__ void k_sell_gather(int ne, const int* __restrict__ map, const double* __restrict__ val,
                              double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) out[e] = map[e] >= 0 ? val[map[e]] : 0.0;
}

// FEM rows of the block-triangular preconditioner: out_i = v_i - sum over the coupling columns
// (>= nv: the surface unknowns) of S_ij z_j, with z_j already preconditioned; columns are sorted,
// so the coupling entries close each row
__global__ void k_couple_sub(int nv, const int* __restrict__ ptr, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ v,
                             const double* __restrict__ z, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double acc = 0.0;
  for (int k = ptr[i + 1] - 1; k >= ptr[i] && col[k] >= nv; --k) acc += val[k] * z[col[k]];
  out[i] = v[i] - acc;
}

// surface rows of the block preconditioner: z = dinv v
__global__ void k_scale_rows(int r0, int r1, const double* __restrict__ v, const double* __restrict__ dinv,
                             double* __restrict__ z) {
  int i = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r1) z[i] = dinv[i] * v[i];
}

__global__ void k_set_rhs(int nm, int col0, double scale, const double* __restrict__ coul, double* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nm) b[col0 + i] = scale * coul[i];
}

__global__ void k_sub_load(int nv, const double* __restrict__ N, double* __restrict__ d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nv) d[i] -= N[i];
}

__global__ void k_trace(int ns, const int* __restrict__ vmap, const double* __restrict__ u, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) out[i] = u[vmap[i]];
}

__global__ void k_div(int n, const double* __restrict__ x, const double* __restrict__ d, double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] / d[i];
}

}  // namespace

// ------------------------------------------------------------------ small BLAS

void timer_begin(Mesh* m, KernelClassTimer& t, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!m->timing) return;
  cudaEventCreate(ev);
  cudaEventRecord(*ev, m->stream);
}

void timer_end(Mesh* m, KernelClassTimer& t, cudaEvent_t ev0, double work) {
  t.count += 1;
  t.work += work;
  if (!m->timing || !ev0) return;
  cudaEvent_t ev1;
  cudaEventCreate(&ev1);
  cudaEventRecord(ev1, m->stream);
  t.pending.push_back({ev0, ev1});
}

void timer_flush(KernelClassTimer& t) {
  for (auto& p : t.pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.second);
    cudaEventElapsedTime(&ms, p.first, p.second);
    t.ms += ms;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  t.pending.clear();
}

int launch_axpby(Mesh* m, int n, double a, const double* x, double b, const double* y, double* z) {
  k_axpby<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, a, x, b, y, z);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

// device dot product into device scalar out_dev
static int dot_dev(Mesh* m, const double* a, const double* b, int n, double* out_dev) {
  int nb = std::min(DOT_B, std::max(1, blocks_for(n, DOT_T)));
  k_dot_partial<<<nb, DOT_T, 0, m->stream>>>(n, a, b, m->red.p);
  PB_LAUNCHED(m);
  k_sum_to<<<1, 32, 0, m->stream>>>(m->red.p, nb, out_dev);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int dot(Mesh* m, const double* a, const double* b, int n, double* out_host) {
  PB_TRY(dot_dev(m, a, b, n, m->scal.p + 4000));
  PB_CUDA(cudaMemcpyAsync(m->pinned, m->scal.p + 4000, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  *out_host = m->pinned[0];
  return PBFB_OK;
}

// ------------------------------------------------------------------ parameters and operator

static int set_params(Mesh* m, double eps_in, double eps_out, double kappa, double T, int precision) {
  if (!(eps_in > 0) || !(eps_out > 0) || !(kappa >= 0) || !(T > 0) || !std::isfinite(kappa) ||
      !std::isfinite(eps_in) || !std::isfinite(eps_out) || !std::isfinite(T)) {
    set_error("invalid parameters: eps_in %g eps_out %g kappa %g T %g", eps_in, eps_out, kappa, T);
    return PBFB_ERR_INVALID;
  }
  if (precision != PBFB_FP64 && precision != PBFB_MIXED && precision != PBFB_FLOAT2) {
    set_error("invalid precision %d", precision);
    return PBFB_ERR_INVALID;
  }
  PB_CUDA(cudaSetDevice(m->dev));
  m->eps_m = eps_in;
  m->eps_s = eps_out;
  m->kappa = kappa;
  m->T = T;
  m->kT = kBoltzmann * T;
  m->lB = kCoulomb / m->kT;
  m->coef = eps_out * kappa * kappa;
  m->precision = precision;
  if (!m->ss.built || m->ss.kappa != kappa) {
    PB_TRY(launch_pair_corrections(m, &m->ss, kappa));
    m->ss.kappa = kappa;
    m->ss.built = true;
  }
  PB_TRY(launch_fill_operator(m));
  PB_CUDA(cudaMemcpyAsync(m->s_val.p, m->s_base.p, m->snnz * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  m->params = true;
  return PBFB_OK;
}

// J(u) into the operator values; N(u) into N_out (may be null)
static int assemble(Mesh* m, int scheme, const double* u, double* N_out) {
  bool ff = false;
  PB_TRY(launch_element_nl(m, scheme, u, m->coef, m->tloc.p, &ff));
  PB_TRY(launch_gather(m, m->snnz, m->jg_ptr.p, m->jg_idx.p, m->tloc.p, m->s_base.p, 1.0, m->s_val.p, ff));
  if (N_out)
    PB_TRY(launch_gather(m, m->nv, m->ng_ptr.p, m->ng_idx.p, m->tloc.p + 10 * m->nt, nullptr, 1.0, N_out, ff));
  return PBFB_OK;
}

static int clear_jacobian(Mesh* m) {
  PB_CUDA(cudaMemcpyAsync(m->s_val.p, m->s_base.p, m->snnz * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return PBFB_OK;
}

// y = Acal(J) x: sparse part, then the far field of both surfaces into their rows, with the
// far field in the given precision
static int apply_prec(Mesh* m, const double* x, double* y, int precision) {
  PB_TRY(launch_spmv(m, x, y));
  Surface* sm = &m->sm;
  Surface* ss = &m->ss;
  // Gamma_m rows: (M/2 + K_L) u - V_L lam_m (the identity when Gamma_m is interior); Gamma_s
  // rows: (M/2 - K_Y) u + V_Y lam_s
  if (!m->full) PB_TRY(launch_bem_far(m, sm, x, x + sm->col0, -1.0, 1.0, 0.0, precision, y + sm->col0, true));
  PB_TRY(launch_bem_far(m, ss, x, x + ss->col0, 1.0, -1.0, m->kappa, precision, y + ss->col0, true));
  return PBFB_OK;
}

static int apply(Mesh* m, const double* x, double* y) { return apply_prec(m, x, y, m->precision); }

int ensure(DBuf<double>& b, size_t n) {
  if (b.n >= n) return PBFB_OK;
  return b.alloc(n);
}

static int ensure_f(DBuf<float>& b, size_t n) {
  if (b.n >= n) return PBFB_OK;
  return b.alloc(n);
}

static int jacobi(Mesh* m, double* dinv) {
  k_jacobi<<<blocks_for(m->n, 256), 256, 0, m->stream>>>(m->nv, m->sm.nv, m->ss.nv, m->s_ptr.p, m->s_col.p,
                                                          m->s_val.p, m->full ? nullptr : m->sm.diagV.p,
                                                          m->ss.diagV.p, dinv);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

// ------------------------------------------------------------------ GMRES

// Block preconditioner z = P(v), block triangular: the surface rows first (z = diag^-1 v, or the
// dense single-layer inverses), then inner_iters Jacobi-PCG iterations from z_u = 0 on
// (A + J) z_u = v_u - S_{u,lam} z_lam, the FEM rows' right-hand side minus their (sparse, mass)
// coupling to the surface unknowns just computed.  Deterministic (fixed reductions, fixed count).
// FEM block of the preconditioner: A + J plus the Robin term eps_s (kappa + 1/R) M_s on Gamma_s
// (the constant mode of the exterior Dirichlet-to-Neumann map of a sphere of Gamma_s's area),
// which keeps it positive definite when J = 0.
// With dense = true the surface rows use the dense float32 inverses of V_L and V_Y (built
// once per mesh, and for Gamma_s again whenever kappa changes) on surfaces of at most
// DENSE_V_MAX vertices, the diagonal otherwise.
// Sliced-ELL pattern of the FEM block (rows < nv, columns < nv) from the host CSR pattern: per slice
// of 32 rows the largest row length, entries stored column by column; map[e] = the CSR slot of entry
// e, or -1 for padding (whose column is the row itself).
static int build_sell(Mesh* m) {
  const int nv = m->nv;
  const int nslice = (nv + 31) / 32;
  std::vector<int> ptr(nslice + 1, 0), col, map;
  for (int sl = 0; sl < nslice; ++sl) {
    int wd = 0;
    for (int r = 32 * sl; r < std::min(nv, 32 * sl + 32); ++r) {
      int c = 0;
      for (int k = m->s_ptr_h[r]; k < m->s_ptr_h[r + 1]; ++k) c += m->s_col_h[k] < nv;
      wd = std::max(wd, c);
    }
    ptr[sl + 1] = ptr[sl] + 32 * wd;
  }
  col.assign(ptr[nslice], 0);
  map.assign(ptr[nslice], -1);
  for (int sl = 0; sl < nslice; ++sl) {
    const int wd = (ptr[sl + 1] - ptr[sl]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int r = 32 * sl + l;
      int j = 0;
      if (r < nv)
        for (int k = m->s_ptr_h[r]; k < m->s_ptr_h[r + 1]; ++k)
          if (m->s_col_h[k] < nv) {
            col[ptr[sl] + 32 * j + l] = m->s_col_h[k];
            map[ptr[sl] + 32 * j + l] = k;
            ++j;
          }
      for (; j < wd; ++j) col[ptr[sl] + 32 * j + l] = r < nv ? r : 0;
    }
  }
  m->sell_nslice = nslice;
  m->sell_ne = ptr[nslice];
  PB_TRY(m->sell_ptr.upload(ptr.data(), ptr.size(), m->stream));
  PB_TRY(m->sell_col.upload(col.data(), col.size(), m->stream));
  PB_TRY(m->sell_map.upload(map.data(), map.size(), m->stream));
  PB_TRY(m->sell_val.alloc(ptr[nslice]));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  m->sell_ok = true;
  return PBFB_OK;
}

static int prepare_block_precond(Mesh* m, bool dense) {
  m->dense_m = dense && !m->full && m->sm.nv <= DENSE_V_MAX;
  m->dense_s = dense && m->ss.nv <= DENSE_V_MAX;
  if (m->dense_m && !m->sm.vinv_ok) PB_TRY(build_dense_single_layer(m, &m->sm, 0.0, true));
  if (m->dense_s && (!m->ss.vinv_ok || m->ss.vinv_kappa != m->kappa))
    PB_TRY(build_dense_single_layer(m, &m->ss, m->kappa, true));
  if (m->no_coop) m->coop_blocks = -1;
  if (m->coop_blocks == 0) {
    int coop = 0, nsm = 0, per = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, m->dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->dev);
    int per4 = 0, per2 = 0;
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_coop<8>, PCG_T, 0));
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per4, k_pcg_coop<4>, PCG_T, 0));
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_pcg_coop<2>, PCG_T, 0));
    int per1 = 0, perf8 = 0, perf4 = 0, perf2 = 0;
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_pcg_coop_sell, PCG_T, 0));
    per = std::min({per, per4, per2, per1});  // co-resident with every variant
    // the float32 form: one block per SM
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perf8, k_pcg_coop_f32<8>, PCG_F32_T, 0));
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perf4, k_pcg_coop_f32<4>, PCG_F32_T, 0));
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perf2, k_pcg_coop_f32<2>, PCG_F32_T, 0));
    m->coop_blocks_f32 = (coop && std::min({perf8, perf4, perf2}) >= 1) ? nsm : -1;
    int perr = 0;
    PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perr, k_pcg_pipe_f32, PCG_PIPE_T, 0));
    m->coop_blocks_pipe = (coop && perr >= 1) ? nsm : 0;
    // all resident blocks (memory-level parallelism for the SpMV phases), but no more than
    // one pass of 8 lanes per row needs
    int want = (m->tune_pcg_bps > 0 ? std::min(per, m->tune_pcg_bps) : per) * nsm;
    want = std::min(want, std::max(1, blocks_for((int64_t)m->nv * 8, PCG_T)));
    m->coop_blocks = (coop && per > 0) ? want : -1;
  }
  PB_TRY(ensure(m->pval, m->fem_nnz));
  PB_TRY(ensure(m->pdinv, m->nv));
  PB_TRY(ensure(m->gpart, 4 * (size_t)std::max({m->coop_blocks, m->coop_blocks_f32, 152}) + 8));
  PB_CUDA(cudaMemcpyAsync(m->pval.p, m->s_val.p, m->fem_nnz * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  const double c = m->eps_s * (m->kappa + 1.0 / m->gs_radius);
  if (m->nrobin) {
    k_add_robin<<<blocks_for(m->nrobin, 256), 256, 0, m->stream>>>(m->nrobin, m->robin_slot.p, m->robin_ref.p,
                                                                    m->ss.mass.p, c, m->pval.p);
    PB_LAUNCHED(m);
  }
  k_diag_inv<<<blocks_for(m->nv, 256), 256, 0, m->stream>>>(m->nv, m->s_ptr.p, m->s_col.p, m->pval.p, m->pdinv.p);
  PB_LAUNCHED(m);
  // the cooperative PCG in float32: by default in the mixed precision (not the sliced-ELL form)
  const int pp = m->tune_pcg_prec;
  m->pcg_f32 = m->coop_blocks > 0 && m->coop_blocks_f32 > 0 && m->pcg_lanes != 1 &&
               (pp == 2 || (pp == 0 && m->precision == PBFB_MIXED));
  if (m->pcg_f32) {
    if (m->pcgf.n < 6 * (size_t)m->n) {
      PB_TRY(m->pcgf.alloc(6 * (size_t)m->n));
      PB_CUDA(cudaMemsetAsync(m->pcgf.p, 0, 6 * (size_t)m->n * sizeof(float), m->stream));
    }

    PB_TRY(ensure_f(m->pvalf, m->fem_nnz));
    PB_TRY(ensure_f(m->pdinvf, m->nv));
    k_to_f32<<<blocks_for(m->fem_nnz, 256), 256, 0, m->stream>>>(m->fem_nnz, m->pval.p, m->pvalf.p);
    PB_LAUNCHED(m);
    k_to_f32<<<blocks_for(m->nv, 256), 256, 0, m->stream>>>(m->nv, m->pdinv.p, m->pdinvf.p);
    PB_LAUNCHED(m);
  }
  if (m->coop_blocks > 0 && m->pcg_lanes == 1) {
    if (!m->sell_ok) PB_TRY(build_sell(m));
    k_sell_gather<<<blocks_for(m->sell_ne, 256), 256, 0, m->stream>>>(m->sell_ne, m->sell_map.p, m->pval.p,
                                                                      m->sell_val.p);
    PB_LAUNCHED(m);
  }
  return PBFB_OK;
}

// Surface rows of the block preconditioner: z_m = (-V_L)^-1 v_m and z_s = V_Y^-1 v_s from the
// dense inverses (the stored matrices are -V^-1), else the diagonal.
static int surface_rows_precond(Mesh* m, const double* v, double* z) {
  const int nv = m->nv, n = m->n, c0 = m->sm.col0, c1 = m->ss.col0;
  if (m->dense_m) {
    PB_TRY(launch_dense_apply(m, &m->sm, 1.0, v + c0, z + c0));
  } else {
    k_scale_rows<<<blocks_for(c1 - c0, 256), 256, 0, m->stream>>>(c0, c1, v, m->gdiag.p, z);
    PB_LAUNCHED(m);
  }
  if (m->dense_s) {
    PB_TRY(launch_dense_apply(m, &m->ss, -1.0, v + c1, z + c1));
  } else {
    k_scale_rows<<<blocks_for(n - c1, 256), 256, 0, m->stream>>>(c1, n, v, m->gdiag.p, z);
    PB_LAUNCHED(m);
  }
  (void)nv;
  return PBFB_OK;
}

// Inner Jacobi-PCG on the FEM block as separate kernels (no grid barrier), then the surface rows.
static int block_precond_launches(Mesh* m, const double* v, double* z, int inner_iters, int nb) {
  const int nv = m->nv, n = m->n;
  double* pb = m->gpcg.p;
  double* pr = pb + (size_t)n;
  double* pz = pb + 2 * (size_t)n;
  double* pp = pb + 3 * (size_t)n;
  double* pq = pb + 4 * (size_t)n;
  double* vu = pb + 8 * (size_t)n;   // FEM right-hand side minus the coupling to z's surface part
  double* part = m->gpart.p;
  double* sc = m->scal.p + 5000;     // [0] pq, [1 + k] rz_k
  const double* dinv = m->pdinv.p;
  PB_TRY(surface_rows_precond(m, v, z));
  k_couple_sub<<<blocks_for(nv, 256), 256, 0, m->stream>>>(nv, m->s_ptr.p, m->s_col.p, m->s_val.p, v, z, vu);
  PB_LAUNCHED(m);
  k_pcg_init<<<nb, PCG_T, 0, m->stream>>>(nv, vu, dinv, z, pr, pz, pp, part);
  PB_LAUNCHED(m);
  k_sum_to<<<1, 32, 0, m->stream>>>(part, nb, sc + 1);
  PB_LAUNCHED(m);
  for (int k = 0; k < inner_iters; ++k) {
    k_pcg_spmv<<<nb, PCG_T, 0, m->stream>>>(nv, m->s_ptr.p, m->s_col.p, m->pval.p, pp, pq, part);
    PB_LAUNCHED(m);
    k_sum_to<<<1, 32, 0, m->stream>>>(part, nb, sc);
    PB_LAUNCHED(m);
    k_pcg_update<<<nb, PCG_T, 0, m->stream>>>(nv, sc + 1 + k, sc, z, pr, pp, pq, dinv, pz, part);
    PB_LAUNCHED(m);
    k_sum_to<<<1, 32, 0, m->stream>>>(part, nb, sc + 2 + k);
    PB_LAUNCHED(m);
    k_pcg_direction<<<nb, PCG_T, 0, m->stream>>>(nv, sc + 1 + k, sc + 2 + k, pz, pp);
    PB_LAUNCHED(m);
  }
  return PBFB_OK;
}

static int block_precond(Mesh* m, const double* v, double* z, int inner_iters) {
  const int nv = m->nv, n = m->n;
  const int nb = std::min(152, std::max(1, blocks_for(nv, PCG_T)));
  double* pb = m->gpcg.p;            // pcg vectors (each n long; surface part of p stays 0)
  double* pr = pb + (size_t)n;
  double* pz = pb + 2 * (size_t)n;
  double* pp = pb + 3 * (size_t)n;
  double* pq = pb + 4 * (size_t)n;
  double* part = m->gpart.p;
  const double* dinv = m->pdinv.p;
  if (m->coop_blocks > 0) {
    // surface rows first, then the FEM block on v_u minus the coupling to them
    PB_TRY(surface_rows_precond(m, v, z));
    double* vu = pb + 8 * (size_t)n;
    k_couple_sub<<<blocks_for(nv, 256), 256, 0, m->stream>>>(nv, m->s_ptr.p, m->s_col.p, m->s_val.p, v, z, vu);
    PB_LAUNCHED(m);
    int nbc = m->coop_blocks, iters = inner_iters, nvv = nv;
    const int* sp = m->s_ptr.p;
    const int* sc2 = m->s_col.p;
    const double* pv = m->pval.p;
    double* pw = pb + 5 * (size_t)n;
    if (m->pcg_lanes == 1 && m->sell_ok) {
      int nsl = m->sell_nslice;
      const int* sp1 = m->sell_ptr.p;
      const int* sc1 = m->sell_col.p;
      const double* sv1 = m->sell_val.p;
      void* args1[] = {&nvv, &nsl, &iters, &sp1, &sc1, &sv1, (void*)&vu, (void*)&dinv, &z, &pr, &pz, &pp, &pq,
                       &pw, &part};
      PB_CUDA(cudaLaunchCooperativeKernel((const void*)k_pcg_coop_sell, dim3(nbc), dim3(PCG_T), args1, 0, m->stream));
      PB_LAUNCHED(m);
      return PBFB_OK;
    }
    if (m->pcg_f32) {
      // float32 vectors, n each: the FEM rows' coupling columns (>= nv) read z there, which stays 0
      float* fx = m->pcgf.p;
      float* fr = fx + (size_t)n;
      float* fz = fx + 2 * (size_t)n;
      float* fp = fx + 3 * (size_t)n;
      float* fq = fx + 4 * (size_t)n;
      float* fw = fx + 5 * (size_t)n;
      const float* fv = m->pvalf.p;
      const float* fd = m->pdinvf.p;
      void* argsf[] = {&nvv, &iters, &sp, &sc2, &fv, (void*)&vu, &fd, &z, &fx, &fr, &fz, &fp, &fq, &fw, &part};
      if (nv <= PCG_RES_ROWS * m->coop_blocks_pipe) {
        int nbr = (nv + PCG_RES_ROWS - 1) / PCG_RES_ROWS;
        float* mb = fx;  // m, two buffers of nv (the x and r vectors of the form below)
        float* ub = fq;
        void* argsr[] = {&nvv, &iters, &sp, &sc2, &fv, (void*)&vu, &fd, &z, &mb, &ub, &part};
        PB_CUDA(cudaLaunchCooperativeKernel((const void*)k_pcg_pipe_f32, dim3(nbr), dim3(PCG_PIPE_T), argsr, 0,
                                            m->stream));
        PB_LAUNCHED(m);
        return PBFB_OK;
      }
      const void* kf = m->pcg_lanes == 2   ? (const void*)k_pcg_coop_f32<2>
                       : m->pcg_lanes == 4 ? (const void*)k_pcg_coop_f32<4>
                                           : (const void*)k_pcg_coop_f32<8>;
      PB_CUDA(cudaLaunchCooperativeKernel(kf, dim3(m->coop_blocks_f32), dim3(PCG_F32_T), argsf, 0, m->stream));
      PB_LAUNCHED(m);
      return PBFB_OK;
    }
    void* args[] = {&nvv, &iters, &sp, &sc2, &pv, (void*)&vu, (void*)&dinv, &z, &pr, &pz, &pp, &pq, &pw, &part};
    const void* kfn = m->pcg_lanes == 2   ? (const void*)k_pcg_coop<2>
                      : m->pcg_lanes == 4 ? (const void*)k_pcg_coop<4>
                                          : (const void*)k_pcg_coop<8>;
    PB_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(nbc), dim3(PCG_T), args, 0, m->stream));
    PB_LAUNCHED(m);
    return PBFB_OK;
  }
  // the ~5 inner_iters + 4 small launches replayed as one CUDA graph on fixed buffers
  double* gin = pb + 6 * (size_t)n;
  double* gout = pb + 7 * (size_t)n;
  const void* key[9] = {m->gpcg.p, m->gpart.p, m->pval.p, m->pdinv.p, m->s_val.p, m->gdiag.p,
                        m->dense_m ? (const void*)m->sm.vinv.p : nullptr,
                        m->dense_s ? (const void*)m->ss.vinv.p : nullptr, m->s_ptr.p};
  if (!m->pcg_graph_off && m->gpcg.n >= 9 * (size_t)n &&
      (!m->pcg_graph || m->pcg_graph_iters != inner_iters || !std::equal(key, key + 9, m->pcg_graph_key))) {
    if (m->pcg_graph) cudaGraphExecDestroy(m->pcg_graph);
    m->pcg_graph = nullptr;
    const double launches0 = m->launches;
    cudaGraph_t g = nullptr;
    int st = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? PBFB_OK : -1;
    if (st == PBFB_OK) {
      st = block_precond_launches(m, gin, gout, inner_iters, nb);
      const cudaError_t e = cudaStreamEndCapture(m->stream, &g);
      if (st == PBFB_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&m->pcg_graph, g, 0) == cudaSuccess) {
        m->pcg_graph_nodes = m->launches - launches0;
        m->pcg_graph_iters = inner_iters;
        std::copy(key, key + 9, m->pcg_graph_key);
      } else {
        m->pcg_graph = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a refused capture leaves no error behind
    m->launches = launches0;
    if (!m->pcg_graph) m->pcg_graph_off = true;
  }
  if (m->pcg_graph) {
    PB_CUDA(cudaMemcpyAsync(gin, v, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    PB_CUDA(cudaGraphLaunch(m->pcg_graph, m->stream));
    PB_CUDA(cudaMemcpyAsync(z, gout, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    m->launches += m->pcg_graph_nodes;
    return PBFB_OK;
  }
  return block_precond_launches(m, v, z, inner_iters, nb);
}

int block_precond_apply(Mesh* m, const double* v, double* z, int inner_iters, bool dense) {
  const int n = m->n;
  PB_TRY(ensure(m->gdiag, n));
  if (m->gpcg.n < 9 * (size_t)n) {
    PB_TRY(m->gpcg.alloc(9 * (size_t)n));
    PB_CUDA(cudaMemsetAsync(m->gpcg.p, 0, 9 * (size_t)n * sizeof(double), m->stream));
  }
  PB_TRY(jacobi(m, m->gdiag.p));
  PB_TRY(prepare_block_precond(m, dense));
  return block_precond(m, v, z, inner_iters);
}

static int gmres(Mesh* m, const double* b, double* x, double tol, int restart, int maxit, int precond,
                 int inner_iters, int* iters_out, double* rel_out) {
  const int n = m->n;
  if (restart < 1 || restart > 400) {
    set_error("restart must be in [1, 400]");
    return PBFB_ERR_INVALID;
  }
  if ((precond != PBFB_PRECOND_JACOBI && precond != PBFB_PRECOND_BLOCK && precond != PBFB_PRECOND_BLOCK_DENSE) ||
      inner_iters < 1 || inner_iters > 500) {
    set_error("invalid preconditioner settings");
    return PBFB_ERR_INVALID;
  }
  const bool flexible = precond != PBFB_PRECOND_JACOBI;
  if (flexible) {
    PB_TRY(ensure(m->gZ, (size_t)restart * n));
    if (m->gpcg.n < 9 * (size_t)n) {
      PB_TRY(m->gpcg.alloc(9 * (size_t)n));
      PB_CUDA(cudaMemsetAsync(m->gpcg.p, 0, 9 * (size_t)n * sizeof(double), m->stream));
    }
  }
  PB_TRY(ensure(m->gV, (size_t)(restart + 1) * n));
  PB_TRY(ensure(m->gw, n));
  PB_TRY(ensure(m->gz, n));
  PB_TRY(ensure(m->gr, n));
  PB_TRY(ensure(m->gdiag, n));
  PB_TRY(ensure(m->gh, 4 * (size_t)(restart + 2)));
  const int nbr = std::min(152, std::max(1, blocks_for(n, MD_T)));
  PB_TRY(ensure(m->gpart, (size_t)(restart + 2) * nbr + 8));
  PB_TRY(jacobi(m, m->gdiag.p));
  if (flexible) PB_TRY(prepare_block_precond(m, precond == PBFB_PRECOND_BLOCK_DENSE));
  if (flexible && m->gones.n < (size_t)n) {
    PB_TRY(m->gones.alloc(n));
    std::vector<double> ones(n, 1.0);
    PB_CUDA(cudaMemcpyAsync(m->gones.p, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    PB_CUDA(cudaStreamSynchronize(m->stream));
  }
  double* V = m->gV.p;
  double* w = m->gw.p;
  double* z = m->gz.p;
  double* r = m->gr.p;
  double* h1 = m->gh.p;                 // restart + 1
  double* h2 = m->gh.p + (restart + 2);  // restart + 1
  double* nrm = m->gh.p + 2 * (restart + 2);
  double* ydev = m->gh.p + 3 * (restart + 2);
  double bn2;
  PB_TRY(dot(m, b, b, n, &bn2));
  double bn = std::sqrt(bn2);
  PB_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), m->stream));
  m->gw_is_ax = false;
  if (iters_out) *iters_out = 0;
  if (rel_out) *rel_out = 0.0;
  if (!(bn > 0)) {
    if (!std::isfinite(bn)) {
      set_error("GMRES: non-finite right-hand side");
      return PBFB_ERR_NONFINITE;
    }
    return PBFB_OK;
  }
  PB_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart);
  std::vector<double> Hraw((size_t)(restart + 1) * restart), u(restart + 1);  // Hessenberg before rotations
  if (m->gones.n < (size_t)n) {
    PB_TRY(m->gones.alloc(n));
    std::vector<double> ones(n, 1.0);
    PB_CUDA(cudaMemcpyAsync(m->gones.p, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    PB_CUDA(cudaStreamSynchronize(m->stream));
  }
  int its = 0, cycle = 0;
  double rel = 1.0;
  double beta = bn;
  while (true) {
    // V[0] = r / ||r||
    PB_TRY(dot_dev(m, r, r, n, nrm));
    k_scale_by<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, r, nrm, V);
    PB_LAUNCHED(m);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (k = 0; k < restart; ++k) {
      double* vk = V + (size_t)k * n;
      if (flexible) {
        double* zk = m->gZ.p + (size_t)k * n;
        PB_TRY(block_precond(m, vk, zk, inner_iters));
        PB_TRY(apply(m, zk, w));
      } else {
        k_mul<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, vk, m->gdiag.p, z);
        PB_LAUNCHED(m);
        PB_TRY(apply(m, z, w));
      }
      // classical Gram-Schmidt, twice
      int kk = k + 1;
      dim3 gd(nbr, (kk + 7) / 8);
      for (int pass = 0; pass < 2; ++pass) {
        double* hh = pass == 0 ? h1 : h2;
        k_multidot<<<gd, MD_T, 0, m->stream>>>(n, kk, V, w, m->gpart.p);
        PB_LAUNCHED(m);
        k_multidot_sum<<<kk, 32, 0, m->stream>>>(m->gpart.p, nbr, kk, hh);
        PB_LAUNCHED(m);
        k_multiaxpy<<<nbr, MD_T, 0, m->stream>>>(n, kk, V, hh, w, pass == 1 ? m->gpart.p : nullptr);
        PB_LAUNCHED(m);
      }
      k_sum_to<<<1, 32, 0, m->stream>>>(m->gpart.p, nbr, nrm);
      PB_LAUNCHED(m);
      k_scale_by<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, w, nrm, V + (size_t)(k + 1) * n);
      PB_LAUNCHED(m);
      // h1 | h2 | nrm are contiguous chunks of gh: one copy
      PB_CUDA(cudaMemcpyAsync(m->pinned, m->gh.p, (2 * (restart + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                              m->stream));
      PB_CUDA(cudaStreamSynchronize(m->stream));
      const double* H1 = m->pinned;
      const double* H2 = m->pinned + (restart + 2);
      double hn = std::sqrt(m->pinned[2 * (restart + 2)]);
      double* col = &H[(size_t)k * (restart + 1)];
      for (int i = 0; i <= k; ++i) col[i] = H1[i] + H2[i];
      col[k + 1] = hn;
      std::copy(col, col + k + 2, &Hraw[(size_t)k * (restart + 1)]);
      for (int i = 0; i < k; ++i) {
        double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      double den = std::hypot(col[k], col[k + 1]);
      if (!std::isfinite(den)) {
        set_error("GMRES: non-finite Arnoldi coefficient");
        return PBFB_ERR_NONFINITE;
      }
      cs[k] = col[k] / den;
      sn[k] = col[k + 1] / den;
      col[k] = den;
      col[k + 1] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++its;
      rel = std::fabs(g[k + 1]) / bn;
      if (rel <= tol || its >= maxit || hn == 0.0) {
        break;
      }
    }
    int mk = std::min(k + 1, restart);
    for (int i = mk - 1; i >= 0; --i) {
      double s = g[i];
      for (int j = i + 1; j < mk; ++j) s -= H[(size_t)j * (restart + 1) + i] * y[j];
      y[i] = s / H[(size_t)i * (restart + 1) + i];
    }
    std::memcpy(m->pinned, y.data(), mk * sizeof(double));
    PB_CUDA(cudaMemcpyAsync(ydev, m->pinned, mk * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    if (flexible) {
      k_update_solution<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, mk, m->gZ.p, ydev, m->gones.p, x);
    } else {
      k_update_solution<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, mk, V, ydev, m->gdiag.p, x);
    }
    PB_LAUNCHED(m);
    if (cycle == 0 && (rel <= tol || its >= maxit)) {
      // done in the first cycle: the Arnoldi relation Acal Z_k = V_{k+1} Hbar_k (flexible) or
      // Acal D V_k = V_{k+1} Hbar_k gives Acal x = V_{k+1} (Hbar_k y) without applying Acal, and the
      // residual norm is the least-squares one, |g_{k+1}| (the operator is deterministic and CGS2
      // keeps the basis orthogonal)
      for (int i = 0; i <= mk; ++i) {
        double t = 0.0;
        for (int j = 0; j < mk; ++j)
          if (i <= j + 1) t += Hraw[(size_t)j * (restart + 1) + i] * y[j];
        u[i] = t;
      }
      // staged through the second half of the pinned buffer: the first half may still be in flight
      std::memcpy(m->pinned + 2048, u.data(), (mk + 1) * sizeof(double));
      double* udev = ydev;  // stream order: the x update above has consumed y already
      PB_CUDA(cudaMemcpyAsync(udev, m->pinned + 2048, (mk + 1) * sizeof(double), cudaMemcpyHostToDevice,
                              m->stream));
      PB_CUDA(cudaMemsetAsync(w, 0, n * sizeof(double), m->stream));
      k_update_solution<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, mk + 1, V, udev, m->gones.p, w);
      PB_LAUNCHED(m);
      PB_CUDA(cudaStreamSynchronize(m->stream));  // both pinned staging areas are reused later
      m->gw_is_ax = true;
      break;
    }
    ++cycle;
    // restart: true residual (w = Acal x stays available to the caller)
    PB_TRY(apply(m, x, w));
    m->gw_is_ax = true;
    PB_TRY(launch_axpby(m, n, 1.0, b, -1.0, w, r));
    double rn2;
    PB_TRY(dot(m, r, r, n, &rn2));
    beta = std::sqrt(rn2);
    rel = beta / bn;
    if (!std::isfinite(rel)) {
      set_error("GMRES: non-finite residual");
      return PBFB_ERR_NONFINITE;
    }
    if (rel <= tol || its >= maxit) break;
  }
  if (iters_out) *iters_out = its;
  if (rel_out) *rel_out = rel;
  if (rel > tol) {
    set_error("GMRES did not converge: relative residual %.3e > %.1e after %d iterations", rel, tol, its);
    return PBFB_ERR_GMRES_NOCONV;
  }
  return PBFB_OK;
}

// ------------------------------------------------------------------ omega evaluation

// Batched a7: dots (host, nomega x 8) = (p+r').r, (p+r').p, (p+r').r', r.r'', p.r'', r.r, p.r, p.p
static int omega_eval(Mesh* m, int scheme, const double* u, const double* du, const double* c, const double* p,
                      const double* omegas, int nomega, double* dots) {
  if (nomega < 1 || nomega > 64) {
    set_error("n_omega must be in [1, 64]");
    return PBFB_ERR_INVALID;
  }
  PB_TRY(ensure(m->wloc, (size_t)nomega * 12 * m->nt));
  // constant (omega-independent) parts over the surface rows, and p.p
  const int nv = m->nv, n = m->n, nb = n - nv;
  double* dv = m->scal.p;  // [0, 64) omegas, [64, ...) results
  std::memcpy(m->pinned, omegas, nomega * sizeof(double));
  PB_CUDA(cudaMemcpyAsync(dv, m->pinned, nomega * sizeof(double), cudaMemcpyHostToDevice, m->stream));
  bool ff = false;
  PB_TRY(launch_omega_elements(m, scheme, u, du, dv, nomega, m->coef, m->wloc.p, &ff));
  PB_TRY(launch_omega_dots(m, nomega, m->wloc.p, c, p, dv + 64, ff));
  PB_TRY(dot_dev(m, p + nv, c + nv, nb, dv + 64 + 7 * 64));
  PB_TRY(dot_dev(m, c + nv, c + nv, nb, dv + 64 + 7 * 64 + 1));
  PB_TRY(dot_dev(m, p, p, n, dv + 64 + 7 * 64 + 2));
  PB_CUDA(cudaMemcpyAsync(m->pinned, dv + 64, (7 * 64 + 3) * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  const double pcb = m->pinned[7 * 64], ccb = m->pinned[7 * 64 + 1], pp = m->pinned[7 * 64 + 2];
  for (int o = 0; o < nomega; ++o) {
    const double* f = m->pinned + 7 * o;  // p.r, r'.r, r'.p, r'.r', r.r'', p.r'', r.r (FEM rows)
    double pr = f[0] + pcb;
    dots[8 * o + 0] = pr + f[1];          // (p+r').r
    dots[8 * o + 1] = pp + f[2];          // (p+r').p
    dots[8 * o + 2] = f[2] + f[3];        // (p+r').r'
    dots[8 * o + 3] = f[4];               // r.r''
    dots[8 * o + 4] = f[5];               // p.r''
    dots[8 * o + 5] = f[6] + ccb;         // r.r
    dots[8 * o + 6] = pr;                 // p.r
    dots[8 * o + 7] = pp;                 // p.p
  }
  return PBFB_OK;
}

static inline double dnorm2(const double* D, double om) { return om * om * D[7] + 2.0 * om * D[6] + D[5]; }

// Fallback of both searches (reading R10): scan g_d(omega) = omega (p+r').p + (p+r').r at
// omega_max j / 16, j = 1..16 (one batched evaluation), bisect its first sign change 20 times,
// accept only if ||d(omega)|| < ||d(0)||.
static int omega_fallback(Mesh* m, int scheme, const double* u, const double* du, const double* c, const double* p,
                          double d0n2, const pbfb_newton_opts& o, double* omega_out, int* evals) {
  double D[8 * 16];
  double om;
  double oms[16];
  for (int j = 0; j < 16; ++j) oms[j] = o.omega_max * (j + 1) / 16.0;
  PB_TRY(omega_eval(m, scheme, u, du, c, p, oms, 16, D));
  ++*evals;
  double lo = 0.0, hi = -1.0;
  for (int j = 0; j < 16; ++j) {
    double gdv = oms[j] * D[8 * j + 1] + D[8 * j + 0];
    if (!std::isfinite(gdv) || gdv >= 0.0) {
      hi = oms[j];
      break;
    }
    lo = oms[j];
  }
  if (hi < 0.0) {
    om = o.omega_max;
  } else {
    for (int it = 0; it < 20; ++it) {
      double mid = 0.5 * (lo + hi);
      PB_TRY(omega_eval(m, scheme, u, du, c, p, &mid, 1, D));
      ++*evals;
      double gdv = mid * D[1] + D[0];
      if (std::isfinite(gdv) && gdv < 0.0)
        lo = mid;
      else
        hi = mid;
    }
    om = 0.5 * (lo + hi);
  }
  PB_TRY(omega_eval(m, scheme, u, du, c, p, &om, 1, D));
  ++*evals;
  double dn = dnorm2(D, om);
  if (!(std::isfinite(dn) && dn < d0n2)) {
    set_error("omega search: no relaxation factor in (0, %g] reduces ||d||", o.omega_max);
    return PBFB_ERR_OMEGA;
  }
  *omega_out = om;
  return PBFB_OK;
}

// Initial guess of the first Newton iteration's omega (Sec. 3.5): three bisection steps of f_d on
// [2, 3] (f_d > 0 moves right), then standard secant steps until |omega_{j+1} - omega_j| < 0.05;
// omega0_first when a value is not finite.
static int warm_start_omega(Mesh* m, int scheme, const double* u, const double* du, const double* c,
                            const double* p, const pbfb_newton_opts& o, double* omega_out, int* evals) {
  double D[8];
  auto fd = [&](double om, double* f) -> int {
    PB_TRY(omega_eval(m, scheme, u, du, c, p, &om, 1, D));
    ++*evals;
    *f = -D[0] / D[1] - om;
    return PBFB_OK;
  };
  double lo = 2.0, hi = 3.0, po[3], pf[3];
  for (int i = 0; i < 3; ++i) {
    double mid = 0.5 * (lo + hi), f;
    PB_TRY(fd(mid, &f));
    po[i] = mid;
    pf[i] = f;
    if (!std::isfinite(f)) {
      *omega_out = o.omega0_first;
      return PBFB_OK;
    }
    if (f > 0.0)
      lo = mid;
    else
      hi = mid;
  }
  double o_prev = po[1], f_prev = pf[1], o_cur = po[2], f_cur = pf[2], o_next = o_cur;
  for (int it = 0; it < o.max_omega_iters; ++it) {
    double den = f_prev - f_cur;
    if (den == 0.0 || !std::isfinite(den)) break;
    o_next = o_prev - (o_prev - o_cur) * f_prev / den;
    if (!std::isfinite(o_next)) {
      o_next = o.omega0_first;
      break;
    }
    if (std::fabs(o_next - o_cur) < 0.05) break;
    o_prev = o_cur;
    f_prev = f_cur;
    o_cur = o_next;
    PB_TRY(fd(o_cur, &f_cur));
    if (!std::isfinite(f_cur)) {
      o_next = o.omega0_first;
      break;
    }
  }
  *omega_out = o_next;
  return PBFB_OK;
}

// Picard relaxation factor: the direct secant of Appendix A (Eq. SEC_FD) through (0, f_d(0) = 1)
// and (omega0, f_d(omega0)), continued by secant steps (Eq. Met_Secante) until |f_d| < Tol_omega;
// accepted under the decrease test, else the shared fallback.
static int picard_omega(Mesh* m, int scheme, const double* u, const double* du, const double* c, const double* p,
                        double d0n2, double omega0, const pbfb_newton_opts& o, double* omega_out, int* evals,
                        int* fallback) {
  double D[8];
  double o_prev = 0.0, f_prev = 1.0, o_cur = omega0;
  PB_TRY(omega_eval(m, scheme, u, du, c, p, &o_cur, 1, D));
  *evals = 1;
  double f_cur = -D[0] / D[1] - o_cur;
  bool ok = false;
  for (int it = 0; it < o.max_omega_iters; ++it) {
    if (!std::isfinite(f_cur)) break;
    if (std::fabs(f_cur) < o.tol_omega) {
      double dn = dnorm2(D, o_cur);
      ok = o_cur > 0.0 && o_cur <= o.omega_max && std::isfinite(dn) && dn < d0n2;
      break;
    }
    double den = f_prev - f_cur;
    if (den == 0.0 || !std::isfinite(den)) break;
    double o_next = o_prev - (o_prev - o_cur) * f_prev / den;
    if (!std::isfinite(o_next)) break;
    o_prev = o_cur;
    f_prev = f_cur;
    o_cur = o_next;
    PB_TRY(omega_eval(m, scheme, u, du, c, p, &o_cur, 1, D));
    ++*evals;
    f_cur = -D[0] / D[1] - o_cur;
  }
  if (ok) {
    *omega_out = o_cur;
    return PBFB_OK;
  }
  PB_TRY(omega_fallback(m, scheme, u, du, c, p, d0n2, o, omega_out, evals));
  ++*fallback;
  return PBFB_OK;
}

static int omega_search(Mesh* m, int scheme, const double* u, const double* du, const double* c, const double* p,
                        double d0n2, double omega0, const pbfb_newton_opts& o, double* omega_out, int* evals,
                        int* fallback) {
  double D[8 * 16];
  double om = omega0;
  bool ok = false;
  *evals = 0;
  for (int it = 0; it < o.max_omega_iters; ++it) {
    PB_TRY(omega_eval(m, scheme, u, du, c, p, &om, 1, D));
    ++*evals;
    double PP = D[1];
    if (!std::isfinite(PP) || std::fabs(PP) < 1e-300) break;
    double f = -D[0] / PP - om;
    double fp = -(D[2] + D[3]) / PP + D[0] * D[4] / (PP * PP) - 1.0;
    if (!std::isfinite(f)) break;
    if (std::fabs(f) < o.tol_omega) {
      double dn = dnorm2(D, om);
      ok = om > 0.0 && om <= o.omega_max && std::isfinite(dn) && dn < d0n2;
      break;
    }
    if (!std::isfinite(fp) || fp == 0.0) break;
    om = om - f / fp;
    if (!std::isfinite(om)) break;
  }
  if (!ok) {
    PB_TRY(omega_fallback(m, scheme, u, du, c, p, d0n2, o, &om, evals));
    ++*fallback;
  }
  *omega_out = om;
  return PBFB_OK;
}

// ------------------------------------------------------------------ energy

// Flux lam on Gamma_m from the trace of u (Sec. 2.3.1): V_L lam = (M_m/2 + K_L) u|Gamma_m
// - c (l_B/eps_m) <u_coul, psi>, c = 1 with the Coulomb term and 0 without.  Flexible
// preconditioned CG on V_L (symmetric positive definite), preconditioned by the dense float32
// V_L^-1 (its diagonal above DENSE_V_MAX vertices), far field in float64 (FP64) or float-float
// (MIXED), to a relative residual of 1e-13.  x is a full vector (only its u part is read); lam
// may alias x's lam_m slots.
static int gamma_m_flux(Mesh* m, const double* x, bool coulomb, double* lam) {
  Surface* s = &m->sm;
  const int nm = s->nv;
  const int prec = m->precision == PBFB_FP64 ? PBFB_FP64 : PBFB_FLOAT2;
  if (coulomb && !m->charges) {
    set_error("Gamma_m flux: charges not set");
    return PBFB_ERR_STATE;
  }
  PB_TRY(ensure(m->pp_val, s->cnnz));
  PB_TRY(ensure(m->pp_work, 7 * (size_t)nm));
  double* rhs = m->pp_work.p;
  double* r = rhs + nm;
  double* z = rhs + 2 * (size_t)nm;
  double* p = rhs + 3 * (size_t)nm;
  double* q = rhs + 4 * (size_t)nm;
  double* ug = rhs + 5 * (size_t)nm;
  double* rold = rhs + 6 * (size_t)nm;
  const bool dense = nm <= DENSE_V_MAX;
  if (dense && !s->vinv_ok) PB_TRY(build_dense_single_layer(m, s, 0.0, true));
  auto precond = [&](const double* v, double* out) -> int {
    if (dense) return launch_dense_apply(m, s, -1.0, v, out);  // the stored matrix is -V^-1
    k_div<<<blocks_for(nm, 256), 256, 0, m->stream>>>(nm, v, s->diagV.p, out);
    PB_LAUNCHED(m);
    return PBFB_OK;
  };
  auto applyV = [&](const double* v, double* out) -> int {
    PB_TRY(launch_bem_far(m, s, v, v, 1.0, 0.0, 0.0, prec, out, false));
    return launch_csr_spmv(m, nm, s->c_ptr.p, s->c_col.p, s->corrV.p, v, out, true);
  };
  // right-hand side
  PB_TRY(launch_axpby(m, s->cnnz, 0.5, s->mass.p, 1.0, s->corrK.p, m->pp_val.p));
  k_trace<<<blocks_for(nm, 256), 256, 0, m->stream>>>(nm, s->vmap.p, x, ug);
  PB_LAUNCHED(m);
  PB_TRY(launch_bem_far(m, s, x, x + s->col0, 0.0, 1.0, 0.0, prec, rhs, false));
  PB_TRY(launch_csr_spmv(m, nm, s->c_ptr.p, s->c_col.p, m->pp_val.p, ug, rhs, true));
  if (coulomb) PB_TRY(launch_axpby(m, nm, 1.0, rhs, -m->lB / m->eps_m, m->coul.p, rhs));
  double bb;
  PB_TRY(dot(m, rhs, rhs, nm, &bb));
  PB_CUDA(cudaMemsetAsync(lam, 0, nm * sizeof(double), m->stream));
  if (!(bb > 0)) {
    if (!std::isfinite(bb)) {
      set_error("Gamma_m flux: non-finite right-hand side");
      return PBFB_ERR_NONFINITE;
    }
    return PBFB_OK;
  }
  PB_CUDA(cudaMemcpyAsync(r, rhs, nm * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  PB_TRY(precond(r, z));
  PB_CUDA(cudaMemcpyAsync(p, z, nm * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  double rz;
  PB_TRY(dot(m, r, z, nm, &rz));
  for (int it = 0; it < 500; ++it) {
    PB_TRY(applyV(p, q));
    double pq;
    PB_TRY(dot(m, p, q, nm, &pq));
    if (!(pq > 0)) break;
    const double alpha = rz / pq;
    PB_TRY(launch_axpby(m, nm, alpha, p, 1.0, lam, lam));
    PB_CUDA(cudaMemcpyAsync(rold, r, nm * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    PB_TRY(launch_axpby(m, nm, -alpha, q, 1.0, r, r));
    double rr;
    PB_TRY(dot(m, r, r, nm, &rr));
    if (!std::isfinite(rr)) break;
    if (rr <= 1e-26 * bb) return PBFB_OK;
    // flexible (Polak-Ribiere) beta: robust to the float32 preconditioner's asymmetry
    PB_TRY(precond(r, z));
    double rz_new, roz;
    PB_TRY(dot(m, r, z, nm, &rz_new));
    PB_TRY(dot(m, rold, z, nm, &roz));
    const double beta = (rz_new - roz) / rz;
    rz = rz_new;
    PB_TRY(launch_axpby(m, nm, 1.0, z, beta, p, p));
  }
  set_error("Gamma_m flux: CG on V_L did not reach a relative residual of 1e-13");
  return PBFB_ERR_GMRES_NOCONV;
}

static int energy(Mesh* m, const double* xL, const double* xNL, double* out4) {
  PB_TRY(ensure(m->tmp, m->n));
  PB_TRY(ensure(m->urb, 2 * (size_t)m->nq));
  PB_TRY(launch_reaction_potentials(m, xL, xNL, m->urb.p));
  std::vector<double> urh(2 * (size_t)m->nq);
  PB_CUDA(cudaMemcpyAsync(urh.data(), m->urb.p, urh.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  // ion term on u = (x_L + x_NL) restricted to the shell
  PB_TRY(launch_axpby(m, m->nv, 1.0, xL, 1.0, xNL, m->tmp.p));
  PB_TRY(launch_ion_energy(m, m->tmp.p, m->scal.p + 1000));
  PB_CUDA(cudaMemcpyAsync(m->pinned, m->scal.p + 1000, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  double LC = 0.0, NC = 0.0;
  for (int k = 0; k < m->nq; ++k) {
    LC += m->qz_h[k] * urh[k];
    NC += m->qz_h[k] * urh[m->nq + k];
  }
  LC *= 0.5 * m->kT;
  NC *= 0.5 * m->kT;
  const double c0 = m->coef / (8.0 * M_PI * m->lB);
  const double dG = m->kT * c0 * m->pinned[0];
  out4[0] = LC + NC + dG;
  out4[1] = LC;
  out4[2] = NC;
  out4[3] = dG;
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(out4[k])) {
      set_error("energy is not finite");
      return PBFB_ERR_NONFINITE;
    }
  return PBFB_OK;
}

// ------------------------------------------------------------------ full solve

static int solve(Mesh* m, double eps_in, double eps_out, double kappa, double T, const pbfb_newton_opts* opts_in,
                 double* x_out_dev, pbfb_result* res) {
  using clk = std::chrono::steady_clock;
  pbfb_newton_opts o;
  pbfb_default_opts(&o);
  if (opts_in) o = *opts_in;
  pbfb_result R;
  std::memset(&R, 0, sizeof(R));
  if (!m->charges) {
    set_error("solve: charges not set");
    return PBFB_ERR_STATE;
  }
  if (!(o.tol_nl > 0) || !(o.tol_gmres > 0) || !(o.tol_gmres0 > 0) || !(o.tol_omega > 0) || o.max_newton < 1 ||
      o.max_gmres < 1 || !(o.omega_max > 0) || !std::isfinite(o.omega_max) || o.max_omega_iters < 1 ||
      !(o.accept_ratio >= 0.0 && o.accept_ratio <= 1.0) || !(o.residual_update >= 0.0) ||
      (o.residual_far != PBFB_FLOAT2 && o.residual_far != PBFB_MIXED) ||
      o.n_taylor < 0 || o.n_taylor > 4 || (o.method != PBFB_NEWTON && o.method != PBFB_PICARD) || !(o.R_e >= 0) ||
      (o.precision != PBFB_FP64 && o.precision != PBFB_MIXED)) {
    set_error("solve: invalid options");
    return PBFB_ERR_INVALID;
  }
  for (int k = 0; k < o.n_taylor; ++k)
    if (o.taylor[k] != PBFB_T3 && o.taylor[k] != PBFB_T5 && o.taylor[k] != PBFB_T7 && o.taylor[k] != PBFB_HS &&
        o.taylor[k] != PBFB_LINEAR) {
      set_error("solve: invalid Taylor schedule entry %d", o.taylor[k]);
      return PBFB_ERR_INVALID;
    }
  PB_TRY(set_params(m, eps_in, eps_out, kappa, T, o.precision));
  const int n = m->n, nv = m->nv;
  for (auto* b : {&m->xL, &m->xNL, &m->phi, &m->cvec, &m->dvec, &m->du, &m->pvec, &m->Nvec, &m->tmp, &m->bvec})
    PB_TRY(ensure(*b, n));
  // right-hand side [0; (l_B/eps_m) <u_coul, psi>; 0], or with Omega_m meshed the point loads
  // [4 pi l_B sum_k z_k v_i(x_k); 0; 0] (Eq. fembem_matrix)
  double* bvec = m->bvec.p;
  PB_CUDA(cudaMemsetAsync(bvec, 0, n * sizeof(double), m->stream));
  if (m->full) {
    PB_TRY(launch_axpby(m, nv, 4.0 * M_PI * m->lB, m->rho.p, 0.0, nullptr, bvec));
  } else {
    k_set_rhs<<<blocks_for(m->sm.nv, 256), 256, 0, m->stream>>>(m->sm.nv, m->sm.col0, m->lB / m->eps_m, m->coul.p,
                                                                 bvec);
    PB_LAUNCHED(m);
  }
  auto t0 = clk::now();
  double tol = o.tol_gmres0;
  // linear part: J = eps_s kappa^2 M (F' = 1)
  PB_CUDA(cudaMemsetAsync(m->phi.p, 0, n * sizeof(double), m->stream));
  PB_TRY(assemble(m, PBFB_LINEAR, m->phi.p, nullptr));
  int its = 0;
  double rel = 0;
  int st = gmres(m, bvec, m->xL.p, tol, o.restart, o.max_gmres, o.precond, o.inner_iters, &its, &rel);
  R.linear_gmres_iters = its;
  if (st) {
    R.status = st;
    if (res) *res = R;
    return st;
  }
  auto t1 = clk::now();
  PB_CUDA(cudaMemsetAsync(m->xNL.p, 0, n * sizeof(double), m->stream));
  double om_last = -1.0, e_prev = -1.0, e_prev2 = -1.0;
  const bool picard = o.method == PBFB_PICARD;
  bool converged = false;
  // residual updates by linearity (residual_update > 0, mixed precision): p of the previous step
  // holds -Acal(0) Delta for its Delta; upd_sum = sum of omega ||Delta|| since the last float-float
  // evaluation of c
  const bool res_upd = o.residual_update > 0.0 && o.precision == PBFB_MIXED;
  bool p_valid = false;
  double upd_sum = 0.0;
  R.residual_updates = 0;
  int k = 0;
  for (k = 0; k < o.max_newton; ++k) {
    const int scheme = k < o.n_taylor ? o.taylor[k] : PBFB_HS;
    PB_TRY(launch_axpby(m, n, 1.0, m->xL.p, 1.0, m->xNL.p, m->phi.p));
    bool updated = false;
    if (res_upd && k > 0 && p_valid) {
      double phi2;
      PB_TRY(dot(m, m->phi.p, m->phi.p, n, &phi2));
      if (upd_sum + e_prev <= o.residual_update * std::sqrt(phi2)) {
        // c_k = c_{k-1} + omega_{k-1} p_{k-1}, p = -Acal(0) Delta_{k-1}
        PB_TRY(launch_axpby(m, n, om_last, m->pvec.p, 1.0, m->cvec.p, m->cvec.p));
        upd_sum += e_prev;
        updated = true;
        ++R.residual_updates;
      }
    }
    if (!updated) {
      // c = b - Acal(0) Phi: the nonlinear residual's far field in float64 (FP64), in float-float
      // or with the GMRES operator's float32 far field (MIXED, residual_far)
      PB_TRY(clear_jacobian(m));
      PB_TRY(apply_prec(m, m->phi.p, m->cvec.p, m->precision == PBFB_MIXED ? o.residual_far : PBFB_FP64));
      PB_TRY(launch_axpby(m, n, 1.0, bvec, -1.0, m->cvec.p, m->cvec.p));
      upd_sum = 0.0;
    }
    p_valid = false;
    // J(u), N(u); d = c - [N; 0; 0]
    PB_TRY(assemble(m, scheme, m->phi.p, m->Nvec.p));
    PB_CUDA(cudaMemcpyAsync(m->dvec.p, m->cvec.p, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    k_sub_load<<<blocks_for(nv, 256), 256, 0, m->stream>>>(nv, m->Nvec.p, m->dvec.p);
    PB_LAUNCHED(m);
    double d2;
    PB_TRY(dot(m, m->dvec.p, m->dvec.p, n, &d2));
    if (!std::isfinite(d2)) {
      set_error("Newton: non-finite residual at iteration %d", k);
      R.status = PBFB_ERR_NONFINITE;
      if (res) *res = R;
      return R.status;
    }
    if (d2 == 0.0) {
      // the iterate solves the system exactly (e.g. no charges): Delta = 0 for every omega, so
      // e_k = 0 < Tol_NL (Sec. 3.5) without a relaxation-factor search
      if (k < PBFB_MAX_TRACE) {
        R.gmres_iters[k] = R.omega_evals[k] = 0;
        R.omega[k] = R.e[k] = 0.0;
      }
      converged = true;
      break;
    }
    // Newton: Acal(J) Delta = d (Eq. NR_main).  Picard: Acal(0) Delta = d, the increment form of
    // Eq. Ec_NL_Previo2 (Delta = Phi~_NL - Phi_NL)
    if (picard) PB_TRY(clear_jacobian(m));
    st = gmres(m, m->dvec.p, m->du.p, tol, o.restart, o.max_gmres, o.precond, o.inner_iters, &its, &rel);
    if (k < PBFB_MAX_TRACE) R.gmres_iters[k] = its;
    if (st) {
      R.status = st;
      R.newton_iters = k + 1;
      if (res) *res = R;
      return st;
    }
    double om;
    int evals = 0;
    // p = -Acal(0) Delta with the GMRES operator (the root of f_d is needed only to Tol_omega):
    // GMRES's final true residual left Acal(J) Delta in gw, and Acal(0) Delta differs from it
    // only by the Jacobian's sparse rows, J Delta = (S_J - S_0) Delta
    auto make_p = [&]() -> int {
      if (m->gw_is_ax) {
        PB_TRY(launch_csr_spmv(m, n, m->s_ptr.p, m->s_col.p, m->s_val.p, m->du.p, m->pvec.p, false));
        PB_TRY(launch_csr_spmv(m, n, m->s_ptr.p, m->s_col.p, m->s_base.p, m->du.p, m->tmp.p, false));
        PB_TRY(launch_axpby(m, n, 1.0, m->pvec.p, -1.0, m->tmp.p, m->pvec.p));
        PB_TRY(launch_axpby(m, n, 1.0, m->pvec.p, -1.0, m->gw.p, m->pvec.p));
        PB_TRY(clear_jacobian(m));
      } else {
        PB_TRY(clear_jacobian(m));
        PB_TRY(apply(m, m->du.p, m->pvec.p));
        PB_TRY(launch_axpby(m, n, -1.0, m->pvec.p, 0.0, nullptr, m->pvec.p));
      }
      p_valid = true;
      return PBFB_OK;
    };
    const bool reuse_newton = !picard && k > 0 && e_prev >= 0.0 && e_prev < o.L_e && om_last > 0.0;
    // R_e rule (Appendix B): keep omega while the error still falls by R_e per step
    const bool reuse_picard = picard && om_last > 0.0 && e_prev2 > 0.0 && e_prev > 0.0 && o.R_e > 0.0 &&
                              !(e_prev2 / e_prev < o.R_e);
    if (!o.omega_search) {
      om = k == 0 ? o.omega0_first : o.omega0_rest;
      if (res_upd) PB_TRY(make_p());
    } else if (reuse_newton || reuse_picard) {
      om = om_last;
      if (res_upd) PB_TRY(make_p());
    } else {
      PB_TRY(make_p());
      double om0 = k == 0 ? o.omega0_first : o.omega0_rest;
      int warm_evals = 0;
      if (k == 0 && o.omega_warm_start && !picard)
        PB_TRY(warm_start_omega(m, scheme, m->phi.p, m->du.p, m->cvec.p, m->pvec.p, o, &om0, &warm_evals));
      // the global convergence condition of Sec. 2.5.2, ||d(omega)|| < ||d(0)||, scaled by accept_ratio
      const double d0n2 = o.accept_ratio * d2;
      st = picard ? picard_omega(m, scheme, m->phi.p, m->du.p, m->cvec.p, m->pvec.p, d0n2, om0, o, &om, &evals,
                                 &R.omega_fallbacks)
                  : omega_search(m, scheme, m->phi.p, m->du.p, m->cvec.p, m->pvec.p, d0n2, om0, o, &om, &evals,
                                 &R.omega_fallbacks);
      evals += warm_evals;
      if (st) {
        R.status = st;
        R.newton_iters = k + 1;
        if (res) *res = R;
        return st;
      }
    }
    om_last = om;
    PB_TRY(launch_axpby(m, n, om, m->du.p, 1.0, m->xNL.p, m->xNL.p));
    double du2;
    PB_TRY(dot(m, m->du.p, m->du.p, n, &du2));
    double e = om * std::sqrt(du2);
    if (k < PBFB_MAX_TRACE) {
      R.omega[k] = om;
      R.e[k] = e;
      R.omega_evals[k] = evals;
    }
    if (!std::isfinite(e)) {
      set_error("Newton: non-finite update at iteration %d", k);
      R.status = PBFB_ERR_NONFINITE;
      if (res) *res = R;
      return R.status;
    }
    e_prev2 = e_prev;
    e_prev = e;
    if (e < 1250.0 * tol) tol = std::max(0.1 * tol, o.tol_gmres);
    if (e < o.tol_nl) {
      converged = true;
      break;
    }
  }
  R.newton_iters = std::min(k + 1, o.max_newton);
  auto t2 = clk::now();
  if (!converged) {
    set_error("%s did not converge in %d iterations", picard ? "Picard" : "Newton", o.max_newton);
    R.status = PBFB_ERR_NEWTON_NOCONV;
    if (res) *res = R;
    return R.status;
  }
  if (m->full) {
    // lam_m from the Gamma_m equation of Sec. 2.3.1, affine in u: the linear part takes the
    // Coulomb term, the nonlinear part none, so that x_L + x_NL carries lam_m of the solution
    PB_TRY(gamma_m_flux(m, m->xL.p, true, m->xL.p + m->sm.col0));
    PB_TRY(gamma_m_flux(m, m->xNL.p, false, m->xNL.p + m->sm.col0));
  }
  double E[4];
  PB_TRY(energy(m, m->xL.p, m->xNL.p, E));
  auto t3 = clk::now();
  R.dG_total = E[0];
  R.dG_LC = E[1];
  R.dG_NC = E[2];
  R.dG_Omega_i = E[3];
  R.ms_linear = std::chrono::duration<double, std::milli>(t1 - t0).count();
  R.ms_newton = std::chrono::duration<double, std::milli>(t2 - t1).count();
  R.ms_energy = std::chrono::duration<double, std::milli>(t3 - t2).count();
  if (x_out_dev) PB_TRY(launch_axpby(m, n, 1.0, m->xL.p, 1.0, m->xNL.p, x_out_dev));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  R.status = PBFB_OK;
  if (res) *res = R;
  return PBFB_OK;
}

int solve_mesh(Mesh* m, double eps_in, double eps_out, double kappa, double T, const pbfb_newton_opts* opts,
               double* x_out_dev, pbfb_result* res) {
  PB_CUDA(cudaSetDevice(m->dev));
  return solve(m, eps_in, eps_out, kappa, T, opts, x_out_dev, res);
}

int charges_set(Mesh* m, const double* xyz, const double* z, int n_q) {
  if (!xyz || !z || n_q < 1) {
    set_error("charges_set: need at least one charge");
    return PBFB_ERR_INVALID;
  }
  std::vector<double> soa(3 * (size_t)n_q);
  for (int k = 0; k < n_q; ++k) {
    for (int d = 0; d < 3; ++d) {
      if (!std::isfinite(xyz[3 * k + d])) {
        set_error("charges_set: non-finite position");
        return PBFB_ERR_INVALID;
      }
      soa[(size_t)d * n_q + k] = xyz[3 * k + d];
    }
    if (!std::isfinite(z[k])) {
      set_error("charges_set: non-finite charge");
      return PBFB_ERR_INVALID;
    }
  }
  if (!m->full) PB_TRY(charges_inside_gamma_m(m, xyz, n_q));
  if (m->full) {
    // point loads of the charges on the Omega_m tets (Eq. fembem_matrix's right-hand side)
    std::vector<double> rho;
    PB_TRY(point_load(m, xyz, z, n_q, rho));
    PB_TRY(m->rho.upload(rho.data(), rho.size(), m->stream));
  }
  PB_TRY(m->qxyz.upload(soa.data(), soa.size(), m->stream));
  PB_TRY(m->qz.upload(z, n_q, m->stream));
  m->qz_h.assign(z, z + n_q);
  m->nq = n_q;
  PB_TRY(m->coul.alloc(m->sm.nv));
  PB_TRY(launch_coulomb(m));
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    set_error("charges_set: %s", cudaGetErrorString(cudaGetLastError()));
    return PBFB_ERR_CUDA;
  }
  m->charges = true;
  return PBFB_OK;
}

void mesh_destroy(Mesh* m) {
  if (!m) return;
  cudaSetDevice(m->dev);
  cudaStreamSynchronize(m->stream);
  timer_flush(m->t_nbody);
  timer_flush(m->t_nbody64);
  timer_flush(m->t_nbodyff);
  timer_flush(m->t_spmv);
  timer_flush(m->t_elem);
  timer_flush(m->t_dense);
  if (m->pinned) cudaFreeHost(m->pinned);
  delete m;
}

}  // namespace pbfb

// ==================================================================== C ABI

using pbfb::Mesh;

struct pbfb_mesh {
  Mesh* m;
};

pbfb::Mesh* pbfb_mesh_internal(pbfb_mesh* h) { return h ? h->m : nullptr; }

#define PB_HANDLE(h)                                  \
  if (!(h) || !(h)->m) {                              \
    pbfb::set_error("null mesh handle");              \
    return PBFB_ERR_INVALID;                          \
  }                                                   \
  Mesh* m = (h)->m;                                   \
  if (cudaSetDevice(m->dev) != cudaSuccess) {         \
    pbfb::set_error("cudaSetDevice failed");          \
    return PBFB_ERR_CUDA;                             \
  }

extern "C" {

void pbfb_default_opts(pbfb_newton_opts* o) {
  if (!o) return;
  o->precision = PBFB_FP64;
  o->tol_nl = 1e-3;
  o->tol_gmres = 1e-6;
  o->tol_gmres0 = 1e-3;
  o->tol_omega = 0.1;
  o->L_e = 0.35;
  o->omega0_first = 2.0;
  o->omega0_rest = 1.0;
  o->omega_max = 4.0;
  o->max_newton = 50;
  o->max_gmres = 1000;
  o->restart = 200;
  o->max_omega_iters = 30;
  o->n_taylor = 1;
  o->taylor[0] = PBFB_T3;
  o->taylor[1] = o->taylor[2] = o->taylor[3] = PBFB_HS;
  o->method = PBFB_NEWTON;
  o->R_e = 1.4;
  o->omega_warm_start = 0;
  o->omega_search = 1;
  o->precond = PBFB_PRECOND_BLOCK_DENSE;
  o->inner_iters = 30;
  o->accept_ratio = 1.0;
  o->residual_update = 0.0;
  o->residual_far = PBFB_FLOAT2;
}

const char* pbfb_last_error(void) { return pbfb::last_error(); }

int pbfb_mesh_create(const double* xyz, int32_t n_v, const int32_t* tets, int64_t n_t, const int32_t* gm_tris,
                     int32_t n_gm, const int32_t* gs_tris, int32_t n_gs, uintptr_t stream, pbfb_mesh** out) {
  pbfb::set_error("");
  if (!out) {
    pbfb::set_error("mesh_create: out is NULL");
    return PBFB_ERR_INVALID;
  }
  *out = nullptr;
  Mesh* m = nullptr;
  int st = pbfb::mesh_create(xyz, n_v, tets, n_t, gm_tris, n_gm, gs_tris, n_gs, (cudaStream_t)stream, &m);
  if (st) return st;
  *out = new pbfb_mesh{m};
  return PBFB_OK;
}

int pbfb_mesh_create_full(const double* xyz, int32_t n_v, const int32_t* tets, int64_t n_t,
                          const int32_t* tet_region, const int32_t* gm_tris, int32_t n_gm, const int32_t* gs_tris,
                          int32_t n_gs, uintptr_t stream, pbfb_mesh** out) {
  pbfb::set_error("");
  if (!out || !tet_region) {
    pbfb::set_error("mesh_create_full: out or tet_region is NULL");
    return PBFB_ERR_INVALID;
  }
  *out = nullptr;
  Mesh* m = nullptr;
  int st = pbfb::mesh_create(xyz, n_v, tets, n_t, gm_tris, n_gm, gs_tris, n_gs, (cudaStream_t)stream, &m,
                             tet_region);
  if (st) return st;
  *out = new pbfb_mesh{m};
  return PBFB_OK;
}

int pbfb_gamma_m_flux(pbfb_mesh* h, const double* x_dev, int coulomb, double* lam_dev) {
  PB_HANDLE(h);
  if (!m->params) {
    pbfb::set_error("call pbfb_set_params first");
    return PBFB_ERR_STATE;
  }
  if (!x_dev || !lam_dev || (coulomb != 0 && coulomb != 1)) {
    pbfb::set_error("gamma_m_flux: bad argument");
    return PBFB_ERR_INVALID;
  }
  int st = pbfb::gamma_m_flux(m, x_dev, coulomb != 0, lam_dev);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_mesh_sizes(const pbfb_mesh* h, int64_t* s) {
  if (!h || !h->m || !s) {
    pbfb::set_error("mesh_sizes: null argument");
    return PBFB_ERR_INVALID;
  }
  const Mesh* m = h->m;
  s[0] = m->nv;
  s[1] = m->nt + m->nt_m;
  s[2] = m->sm.nv;
  s[3] = m->ss.nv;
  s[4] = m->n;
  s[5] = m->fem_nnz;
  s[6] = m->s_ptr_h[m->ss.col0] - m->s_ptr_h[m->sm.col0];
  s[7] = m->s_ptr_h[m->n] - m->s_ptr_h[m->ss.col0];
  return PBFB_OK;
}

int pbfb_surface_vertices(const pbfb_mesh* h, int which, int32_t* out) {
  if (!h || !h->m || !out || (which != PBFB_GAMMA_M && which != PBFB_GAMMA_S)) {
    pbfb::set_error("surface_vertices: bad argument");
    return PBFB_ERR_INVALID;
  }
  const pbfb::Surface& s = which == PBFB_GAMMA_M ? h->m->sm : h->m->ss;
  std::memcpy(out, s.vmap_h.data(), s.vmap_h.size() * sizeof(int32_t));
  return PBFB_OK;
}

int pbfb_charges_set(pbfb_mesh* h, const double* xyz, const double* z, int32_t n_q) {
  PB_HANDLE(h);
  return pbfb::charges_set(m, xyz, z, n_q);
}

int pbfb_solve_device(pbfb_mesh* h, double eps_in, double eps_out, double kappa, double T,
                      const pbfb_newton_opts* opts, double* x_out_dev, pbfb_result* res) {
  PB_HANDLE(h);
  return pbfb::solve(m, eps_in, eps_out, kappa, T, opts, x_out_dev, res);
}

int pbfb_solve(pbfb_mesh* h, double eps_in, double eps_out, double kappa, double T, const pbfb_newton_opts* opts,
               double* u_out, double* lam_m_out, double* lam_s_out, pbfb_result* res) {
  PB_HANDLE(h);
  int st = pbfb::ensure(m->xout, m->n);
  if (st) return st;
  pbfb::DBuf<double>& x = m->xout;
  st = pbfb::solve(m, eps_in, eps_out, kappa, T, opts, x.p, res);
  if (st) return st;
  if (u_out && cudaMemcpy(u_out, x.p, m->nv * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) st = PBFB_ERR_CUDA;
  if (lam_m_out && cudaMemcpy(lam_m_out, x.p + m->sm.col0, m->sm.nv * sizeof(double), cudaMemcpyDeviceToHost))
    st = PBFB_ERR_CUDA;
  if (lam_s_out && cudaMemcpy(lam_s_out, x.p + m->ss.col0, m->ss.nv * sizeof(double), cudaMemcpyDeviceToHost))
    st = PBFB_ERR_CUDA;
  if (st) pbfb::set_error("solve: copy of the solution failed");
  return st;
}

int pbfb_mesh_destroy(pbfb_mesh* h) {
  if (!h) return PBFB_OK;
  pbfb::mesh_destroy(h->m);
  delete h;
  return PBFB_OK;
}

int pbfb_set_params(pbfb_mesh* h, double eps_in, double eps_out, double kappa, double T, int precision) {
  PB_HANDLE(h);
  int st = pbfb::set_params(m, eps_in, eps_out, kappa, T, precision);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

#define PB_NEED_PARAMS                              \
  if (!m->params) {                                 \
    pbfb::set_error("call pbfb_set_params first");  \
    return PBFB_ERR_STATE;                          \
  }

int pbfb_assemble(pbfb_mesh* h, int scheme, const double* u_dev, double* N_out_dev) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!u_dev || scheme < PBFB_LINEAR || scheme > PBFB_T7) {
    pbfb::set_error("assemble: bad argument");
    return PBFB_ERR_INVALID;
  }
  int st = pbfb::assemble(m, scheme, u_dev, N_out_dev);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_clear_jacobian(pbfb_mesh* h) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  int st = pbfb::clear_jacobian(m);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_apply(pbfb_mesh* h, const double* x_dev, double* y_dev) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!x_dev || !y_dev || x_dev == y_dev) {
    pbfb::set_error("apply: bad pointers");
    return PBFB_ERR_INVALID;
  }
  int st = pbfb::apply(m, x_dev, y_dev);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_bem_apply(pbfb_mesh* h, int which, int op, const double* x_dev, double* y_dev) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!x_dev || !y_dev || (which != PBFB_GAMMA_M && which != PBFB_GAMMA_S) || (op != 0 && op != 1)) {
    pbfb::set_error("bem_apply: bad argument");
    return PBFB_ERR_INVALID;
  }
  pbfb::Surface* s = which == PBFB_GAMMA_M ? &m->sm : &m->ss;
  double kap = which == PBFB_GAMMA_M ? 0.0 : m->kappa;
  int st = pbfb::launch_bem_far(m, s, x_dev, x_dev, op == 0 ? 1.0 : 0.0, op == 1 ? 1.0 : 0.0, kap, m->precision,
                                y_dev, false);
  if (st) return st;
  // near-field correction: y += C x (CSR on the surface pattern)
  st = pbfb::launch_csr_spmv(m, s->nv, s->c_ptr.p, s->c_col.p, op == 0 ? s->corrV.p : s->corrK.p, x_dev, y_dev,
                             true);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_single_layer_dense(pbfb_mesh* h, int which, int inverse, float* out_dev, int32_t ld_out) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  pbfb::Surface* s = which == PBFB_GAMMA_M ? &m->sm : &m->ss;
  if (!out_dev || (which != PBFB_GAMMA_M && which != PBFB_GAMMA_S) || (inverse != 0 && inverse != 1) ||
      ld_out < s->nv) {
    pbfb::set_error("single_layer_dense: bad argument");
    return PBFB_ERR_INVALID;
  }
  const double kap = which == PBFB_GAMMA_M ? 0.0 : m->kappa;
  const bool have = s->vinv_ok && s->vinv_kappa == kap;
  if (!inverse || !have) PB_TRY(pbfb::build_dense_single_layer(m, s, kap, inverse != 0));
  // the stored inverse is -V^-1
  PB_TRY(pbfb::dense_copy_out(m, s, inverse ? -1.f : 1.f, out_dev, ld_out));
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_bem_apply_noalloc(pbfb_mesh* h, int which, int op, const double* x_dev, double* y_dev) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!x_dev || !y_dev || x_dev == y_dev || (which != PBFB_GAMMA_M && which != PBFB_GAMMA_S) ||
      (op != 0 && op != 1)) {
    pbfb::set_error("bem_apply_noalloc: bad argument");
    return PBFB_ERR_INVALID;
  }
  int st = pbfb::bem_apply_noalloc(m, which, op, x_dev, y_dev);
  if (st) return st;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? PBFB_OK : PBFB_ERR_CUDA;
}

int pbfb_fem_rows(const pbfb_mesh* h, int32_t* rowptr, int32_t* col, double* val) {
  if (!h || !h->m || !rowptr || !col || !val) {
    pbfb::set_error("fem_rows: null argument");
    return PBFB_ERR_INVALID;
  }
  const Mesh* m = h->m;
  cudaSetDevice(m->dev);
  cudaStreamSynchronize(m->stream);
  std::memcpy(rowptr, m->s_ptr_h.data(), (m->nv + 1) * sizeof(int32_t));
  std::memcpy(col, m->s_col_h.data(), m->fem_nnz * sizeof(int32_t));
  if (cudaMemcpy(val, m->s_val.p, m->fem_nnz * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
    pbfb::set_error("fem_rows: copy failed");
    return PBFB_ERR_CUDA;
  }
  return PBFB_OK;
}

int pbfb_gmres(pbfb_mesh* h, const double* b_dev, double* x_dev, double tol, int restart, int maxit, int precond,
               int inner_iters, int* iters, double* relres) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!b_dev || !x_dev || !(tol > 0) || maxit < 1) {
    pbfb::set_error("gmres: bad argument");
    return PBFB_ERR_INVALID;
  }
  int it = 0;
  double rel = 0;
  int st = pbfb::gmres(m, b_dev, x_dev, tol, restart, maxit, precond, inner_iters, &it, &rel);
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return st;
}

int pbfb_omega_eval(pbfb_mesh* h, int scheme, const double* u_dev, const double* du_dev, const double* c_dev,
                    const double* p_dev, const double* omegas, int n_omega, double* dots) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!u_dev || !du_dev || !c_dev || !p_dev || !omegas || !dots || scheme < PBFB_LINEAR || scheme > PBFB_T7) {
    pbfb::set_error("omega_eval: bad argument");
    return PBFB_ERR_INVALID;
  }
  return pbfb::omega_eval(m, scheme, u_dev, du_dev, c_dev, p_dev, omegas, n_omega, dots);
}

int pbfb_energy(pbfb_mesh* h, const double* xL_dev, const double* xNL_dev, double* out) {
  PB_HANDLE(h);
  PB_NEED_PARAMS;
  if (!m->charges || !xL_dev || !xNL_dev || !out) {
    pbfb::set_error("energy: need charges and vectors");
    return PBFB_ERR_STATE;
  }
  return pbfb::energy(m, xL_dev, xNL_dev, out);
}

int pbfb_set_tuning(pbfb_mesh* h, int nbody_targets_per_thread, int nbody_blocks_per_sm, int nbody_packed) {
  PB_HANDLE(h);
  if (nbody_packed < 0 || nbody_packed > 3) {
    pbfb::set_error("set_tuning: packed must be in 0..3");
    return PBFB_ERR_INVALID;
  }
  m->tune_packed = nbody_packed & 1;
  m->tune_ff_kernel = ((nbody_packed >> 1) & 1) ? 1 : 0;
  if (nbody_targets_per_thread != 0 && nbody_targets_per_thread != 1 && nbody_targets_per_thread != 2 &&
      nbody_targets_per_thread != 4 && nbody_targets_per_thread != 8) {
    pbfb::set_error("set_tuning: targets per thread must be 0, 1, 2, 4 or 8");
    return PBFB_ERR_INVALID;
  }
  if (nbody_blocks_per_sm < 0 || nbody_blocks_per_sm > 64) {
    pbfb::set_error("set_tuning: blocks per SM must be in [0, 64]");
    return PBFB_ERR_INVALID;
  }
  m->tune_tpt = nbody_targets_per_thread;
  m->tune_bps = nbody_blocks_per_sm;
  return PBFB_OK;
}

int pbfb_profile(pbfb_mesh* h, int enable, int reset, double* stats) {
  PB_HANDLE(h);
  cudaStreamSynchronize(m->stream);
  pbfb::timer_flush(m->t_nbody);
  pbfb::timer_flush(m->t_nbody64);
  pbfb::timer_flush(m->t_nbodyff);
  pbfb::timer_flush(m->t_spmv);
  pbfb::timer_flush(m->t_elem);
  pbfb::timer_flush(m->t_dense);
  if (stats) {
    stats[0] = m->launches;
    stats[1] = m->t_nbody.count;
    stats[2] = m->t_nbody.ms;
    stats[3] = m->t_nbody.work;
    stats[4] = m->t_spmv.count;
    stats[5] = m->t_spmv.ms;
    stats[6] = m->t_elem.count;
    stats[7] = m->t_elem.ms;
    stats[8] = m->nbody_flops;
    stats[9] = m->t_nbody64.count;
    stats[10] = m->t_nbody64.ms;
    stats[11] = m->t_nbody64.work;
    stats[12] = m->t_nbodyff.count;
    stats[13] = m->t_nbodyff.ms;
    stats[14] = m->t_nbodyff.work;
    stats[15] = m->t_dense.ms;
    for (int k = 0; k < 4; ++k) stats[16 + k] = m->setup_ms[k];
  }
  if (reset) {
    m->launches = 0;
    m->nbody_flops = 0.0;
    for (auto* t : {&m->t_nbody, &m->t_nbody64, &m->t_nbodyff, &m->t_spmv, &m->t_elem, &m->t_dense}) {
      t->ms = 0;
      t->count = 0;
      t->work = 0;
    }
  }
  m->timing = enable != 0;
  return PBFB_OK;
}

}  // extern "C"
