// Element kernels of the FEM block on the solvent shell Omega_i.
//
// Quantities (weak form of Sec. 2.2, operator split of Eqs. general_nonlinear /
// Vector_c, Jacobian of Eq. NR_main, second derivative of Appendix A):
//   N(u)_i       = eps_s kappa^2 int F(u_h) v_i
//   J(u)_ij      = eps_s kappa^2 int F'(u_h) v_i v_j
//   N''[d,d]_i   = eps_s kappa^2 int F''(u_h) d_h^2 v_i
// with F = u (linear), u + u^3/6 (T3) or sinh u (HS), 14-point rule per tet.
//
// Assembly is deterministic and atomic-free: one thread per tetrahedron writes
// its local values to tet-local storage (structure of arrays, coalesced), and
// a gather kernel sums, for every CSR slot or vertex, a fixed list of those
// entries in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "pbfb_internal.cuh"
#include "quad_tables.cuh"

namespace pbfb {

namespace {

__device__ __forceinline__ void scheme_F(int scheme, double u, double& F, double& Fp, double& Fpp) {
  if (scheme == PBFB_LINEAR) {
    F = u;
    Fp = 1.0;
    Fpp = 0.0;
  } else if (scheme == PBFB_T3 || scheme == PBFB_T5 || scheme == PBFB_T7) {
    // Taylor polynomials of sinh: F = sum u^(2j+1)/(2j+1)!, F' = sum u^(2j)/(2j)!, F'' = F of one degree less
    const double u2 = u * u;
    const int deg = scheme == PBFB_T3 ? 3 : (scheme == PBFB_T5 ? 5 : 7);
    double term_odd = u, term_even = 1.0;  // u^(2j+1)/(2j+1)!, u^(2j)/(2j)!
    F = u;
    Fp = 1.0;
    Fpp = 0.0;
    for (int k = 3; k <= deg; k += 2) {
      Fpp += term_odd;                            // F'' gets the odd terms up to degree deg-2
      term_even *= u2 / ((k - 2) * (k - 1));      // u^(k-1)/(k-1)!
      term_odd *= u2 / ((k - 1) * k);             // u^k/k!
      F += term_odd;
      Fp += term_even;
    }
  } else {
    double e = exp(u);
    double ei = 1.0 / e;
    F = 0.5 * (e - ei);
    Fp = 0.5 * (e + ei);
    Fpp = F;
  }
}

// exp(u) and exp(-u) on the float32 pipes (the mixed precision's sinh / cosh; GB300's float64
// rate is 1/64 of its float32 rate).  Float-float arithmetic (pairs hi + lo of float32 values,
// error-free sums and FMA products, Ogita, Rump & Oishi 2005), about 1e-13 relative:
//   u = m ln2 + r, |r| <= ln2 / 2, with ln2 = L1 + L2 + L3 (L1 of 16 significant bits, so m L1 is
//   exact for |m| <= 128 and u_hi - m L1 exact by Sterbenz' lemma);
//   r = j / 32 + f, |f| <= 1/64;  e^{+-f} = A +- B with the even and odd parts of the series,
//   A = 1 + f^2/2 + f^4/24 + f^6/720 and B = f (1 + f^2/6 + f^4/120 + f^6/5040) (truncation < 1e-17);
//   e^{+-u} = 2^{+-m} e^{+-j/32} (A +- B), the e^{j/32} (|j| <= 12) from a float-float table.
// Used for |u| <= 80 (2^m within float range); larger arguments take the float64 exp.
struct f2 { float h, l; };
__device__ __forceinline__ f2 f2_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_two(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = f2_two(a.h, b.h);
  return f2_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return f2_fast(p, e);
}

constexpr int FX_J = 12;  // table of e^{j/32}, j = -12..12

__device__ __forceinline__ void exp_pm(double u, const float2* __restrict__ tab, double& ep, double& em) {
  if (!(fabs(u) <= 80.0)) {
    ep = exp(u);
    em = exp(-u);
    return;
  }
  constexpr float L1 = 0.693145751953125f;                  // 45426 / 65536
  constexpr float L2 = 1.42860682030941723212e-06f;         // (ln 2 - L1) rounded to float
  constexpr double L3d = 0.69314718055994530942 - 0.693145751953125 - (double)1.42860682030941723212e-06f;
  const float uh = (float)u, ul = (float)(u - (double)uh);
  const float mf = rintf(__fmul_rn(uh, 1.44269504088896340736f));
  // r = u - m (L1 + L2 + L3) in float-float
  f2 r = f2_two(__fsub_rn(uh, __fmul_rn(mf, L1)), ul);
  const float p2 = __fmul_rn(mf, L2), e2 = __fmaf_rn(mf, L2, -p2);
  r = f2_add(r, f2{-p2, -e2});
  r = f2_add(r, f2{-(float)(mf * L3d), 0.f});
  const float jf = rintf(__fmul_rn(r.h, 32.f));
  const f2 f = f2_two(__fsub_rn(r.h, __fmul_rn(jf, 0.03125f)), r.l);
  const f2 s = f2_mul(f, f);
  // A = 1 + s/2 + s^2 (1/24 + s/720)
  const float sa = __fmul_rn(__fmul_rn(s.h, s.h), __fmaf_rn(s.h, 1.f / 720.f, 1.f / 24.f));
  const f2 A = f2_fast(1.f, 0.f);
  const f2 Ah = f2_add(A, f2{__fmul_rn(0.5f, s.h), __fmaf_rn(0.5f, s.l, sa)});
  // B = f (1 + s/6 + s^2 (1/120 + s/5040))
  const float sb = __fmul_rn(__fmul_rn(s.h, s.h), __fmaf_rn(s.h, 1.f / 5040.f, 1.f / 120.f));
  const float s6 = __fmul_rn(s.h, 1.f / 6.f);
  const f2 q = f2_fast(1.f, __fadd_rn(s6, __fadd_rn(__fmaf_rn(s.h, 1.f / 6.f, -s6), __fmaf_rn(s.l, 1.f / 6.f, sb))));
  const f2 B = f2_mul(f, q);
  const f2 Ep = f2_add(Ah, B), Em = f2_add(Ah, f2{-B.h, -B.l});
  const int j = (int)jf + FX_J, m = (int)mf;
  const float2 tp = tab[j], tm = tab[2 * FX_J - j];
  const f2 Pp = f2_mul(Ep, f2{tp.x, tp.y}), Pm = f2_mul(Em, f2{tm.x, tm.y});
  ep = ldexp((double)Pp.h + (double)Pp.l, m);
  em = ldexp((double)Pm.h + (double)Pm.l, -m);
}

// F, F', F'' of the sinh scheme from exp_pm (the other schemes as scheme_F)
__device__ __forceinline__ void scheme_F_fx(int scheme, double u, const float2* __restrict__ tab, double& F,
                                            double& Fp, double& Fpp) {
  if (scheme != PBFB_HS) {
    scheme_F(scheme, u, F, Fp, Fpp);
    return;
  }
  double ep, em;
  exp_pm(u, tab, ep, em);
  F = 0.5 * (ep - em);
  Fp = 0.5 * (ep + em);
  Fpp = F;
}

__global__ void k_tet_volumes(const double* __restrict__ xyz, int nv, const int* __restrict__ tets,
                              int64_t nt, double* __restrict__ vol) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[4];
  for (int a = 0; a < 4; ++a) v[a] = tets[a * nt + t];
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) e[k][d] = xyz[d * nv + v[k + 1]] - xyz[d * nv + v[0]];
  double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
               e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
               e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  vol[t] = fabs(det) / 6.0;
}

// int grad l_a . grad l_b over the tet, 10 symmetric entries at k * nt + t.
__global__ void k_stiffness_local(const double* __restrict__ xyz, int nv, const int* __restrict__ tets,
                                  int64_t nt, const double* __restrict__ vol, double* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[4];
  for (int a = 0; a < 4; ++a) v[a] = tets[a * nt + t];
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) e[k][d] = xyz[d * nv + v[k + 1]] - xyz[d * nv + v[0]];
  // rows of E^{-1}^T: gradient of l_{k+1} = (cofactor row k) / det
  double c[3][3];
  c[0][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
  c[0][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
  c[0][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
  c[1][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
  c[1][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
  c[1][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
  c[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
  c[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
  c[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
  double g[4][3];
  for (int d = 0; d < 3; ++d) {
    g[1][d] = c[0][d] / det;
    g[2][d] = c[1][d] / det;
    g[3][d] = c[2][d] / det;
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  double V = vol[t];
  for (int a = 0; a < 4; ++a)
    for (int b = a; b < 4; ++b)
      loc[(int64_t)sym10(a, b) * nt + t] = V * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
}

__global__ void k_gather(int nslots, const int* __restrict__ ptr, const int* __restrict__ idx,
                         const double* __restrict__ local, const double* __restrict__ base, double scale,
                         double* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslots) return;
  double acc = 0.0;
  for (int k = ptr[s]; k < ptr[s + 1]; ++k) acc += local[idx[k]];
  out[s] = (base ? base[s] : 0.0) + scale * acc;
}

// Jacobian (10 entries, k = 0..9) and load (4 entries, k = 10..13) of F on one tet.
template <bool FX>
__global__ void k_element_nl(int scheme, const double* __restrict__ u, const int* __restrict__ tets, int64_t nt,
                             const double* __restrict__ vol, double coef, const float2* __restrict__ tab,
                             double* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ua[4];
  for (int a = 0; a < 4; ++a) ua[a] = u[tets[a * nt + t]];
  double J[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double N[4] = {0, 0, 0, 0};
  for (int q = 0; q < QT; ++q) {
    double l0 = c_tet_l[q][0], l1 = c_tet_l[q][1], l2 = c_tet_l[q][2], l3 = c_tet_l[q][3];
    double uq = l0 * ua[0] + l1 * ua[1] + l2 * ua[2] + l3 * ua[3];
    double F, Fp, Fpp;
    if (FX)
      scheme_F_fx(scheme, uq, tab, F, Fp, Fpp);
    else
      scheme_F(scheme, uq, F, Fp, Fpp);
    double w = c_tet_w[q];
    double f = w * F, g = w * Fp;
    double l[4] = {l0, l1, l2, l3};
    for (int a = 0; a < 4; ++a) {
      N[a] += f * l[a];
      double gl = g * l[a];
      for (int b = a; b < 4; ++b) J[sym10(a, b)] += gl * l[b];
    }
  }
  double s = coef * vol[t];
  for (int k = 0; k < 10; ++k) loc[k * nt + t] = s * J[k];
  for (int a = 0; a < 4; ++a) loc[(10 + a) * nt + t] = s * N[a];
}

// Sparse part of the coupled operator: y = S x, L lanes per row (L = 4, 8 or 16).
template <int L>
__global__ void k_spmv(int nrows, const int* __restrict__ ptr, const int* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  int lane = threadIdx.x & (L - 1);
  int row = (blockIdx.x * blockDim.x + threadIdx.x) / L;
  const bool valid = row < nrows;  // all lanes reach the shuffles
  double acc = 0.0;
  if (valid)
    for (int k = ptr[row] + lane; k < ptr[row + 1]; k += L) acc += val[k] * __ldg(&x[col[k]]);
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, L);
  if (lane == 0 && valid) y[row] = acc;
}

// Generic CSR y (+)= A x, 8 lanes per row.
__global__ void k_csr_acc(int nrows, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                          int accumulate) {
  int lane = threadIdx.x & 7;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const bool valid = row < nrows;  // all lanes reach the shuffles
  double acc = 0.0;
  if (valid)
    for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 8) acc += val[k] * x[col[k]];
  acc += __shfl_down_sync(0xffffffffu, acc, 4, 8);
  acc += __shfl_down_sync(0xffffffffu, acc, 2, 8);
  acc += __shfl_down_sync(0xffffffffu, acc, 1, 8);
  if (lane == 0 && valid) y[row] = accumulate ? y[row] + acc : acc;
}

// Omega batch: per tet and omega, local load of F(w), of F'(w) du and of F''(w) du^2 at
// w = u + omega du; layout ((o * 3 + quantity) * 4 + a) * nt + t.
template <bool FX>
__global__ void k_omega_elements(int scheme, const double* __restrict__ u, const double* __restrict__ du,
                                 const double* __restrict__ omegas, int nomega, const int* __restrict__ tets,
                                 int64_t nt, const double* __restrict__ vol, double coef,
                                 const float2* __restrict__ tab, double* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ua[4], da[4];
  for (int a = 0; a < 4; ++a) {
    int v = tets[a * nt + t];
    ua[a] = u[v];
    da[a] = du[v];
  }
  double s = coef * vol[t];
  for (int o = 0; o < nomega; ++o) {
    double om = omegas[o];
    double R0[4] = {0, 0, 0, 0}, R1[4] = {0, 0, 0, 0}, R2[4] = {0, 0, 0, 0};
    for (int q = 0; q < QT; ++q) {
      double l[4] = {c_tet_l[q][0], c_tet_l[q][1], c_tet_l[q][2], c_tet_l[q][3]};
      double uq = l[0] * ua[0] + l[1] * ua[1] + l[2] * ua[2] + l[3] * ua[3];
      double dq = l[0] * da[0] + l[1] * da[1] + l[2] * da[2] + l[3] * da[3];
      double F, Fp, Fpp;
      if (FX)
        scheme_F_fx(scheme, uq + om * dq, tab, F, Fp, Fpp);
      else
        scheme_F(scheme, uq + om * dq, F, Fp, Fpp);
      double w = c_tet_w[q];
      double f0 = w * F, f1 = w * Fp * dq, f2 = w * Fpp * dq * dq;
      for (int a = 0; a < 4; ++a) {
        R0[a] += f0 * l[a];
        R1[a] += f1 * l[a];
        R2[a] += f2 * l[a];
      }
    }
    int64_t base = (int64_t)o * 12 * nt;
    for (int a = 0; a < 4; ++a) {
      loc[base + (0 * 4 + a) * nt + t] = s * R0[a];
      loc[base + (1 * 4 + a) * nt + t] = s * R1[a];
      loc[base + (2 * 4 + a) * nt + t] = s * R2[a];
    }
  }
}

constexpr int RED_T = 256;

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* out) {
  __shared__ double sh[RED_T / 32][NV];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double x = 0.0;
    for (int w = 0; w < RED_T / 32; ++w) x += sh[w][threadIdx.x];
    out[threadIdx.x] = x;
  }
}

// Per vertex: gather N(w), J(w) du, N''(w)[du,du] for one omega and accumulate the
// seven FEM-row dot products; one partial row of 7 per block.
__global__ void __launch_bounds__(RED_T) k_omega_dots(int nv, const int* __restrict__ ptr, const int* __restrict__ idx,
                                                      const double* __restrict__ loc, int64_t nt,
                                                      const double* __restrict__ c, const double* __restrict__ p,
                                                      double* __restrict__ part) {
  int o = blockIdx.y;
  const double* L = loc + (int64_t)o * 12 * nt;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * RED_T + threadIdx.x; i < nv; i += gridDim.x * RED_T) {
    double n0 = 0, n1 = 0, n2 = 0;
    for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
      int e = idx[k];
      n0 += L[e];
      n1 += L[4 * nt + e];
      n2 += L[8 * nt + e];
    }
    double r = c[i] - n0, rp = -n1, rpp = -n2, pi = p[i];
    acc[0] += pi * r;     // p.r
    acc[1] += rp * r;     // r'.r
    acc[2] += rp * pi;    // r'.p
    acc[3] += rp * rp;    // r'.r'
    acc[4] += r * rpp;    // r.r''
    acc[5] += pi * rpp;   // p.r''
    acc[6] += r * r;      // r.r
  }
  block_reduce_store<7>(acc, part + ((int64_t)o * gridDim.x + blockIdx.x) * 7);
}

// Sum nb partial rows of width w (for each of gridDim.x problems), fixed order.
__global__ void k_sum_partials(const double* __restrict__ part, int nb, int w, double* __restrict__ out) {
  int o = blockIdx.x;
  for (int k = threadIdx.x; k < w; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[((int64_t)o * nb + b) * w + k];
    out[o * w + k] = s;
  }
}

__global__ void __launch_bounds__(RED_T) k_ion_energy(const double* __restrict__ u, const int* __restrict__ tets,
                                                      int64_t nt, const double* __restrict__ vol,
                                                      double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int64_t t = blockIdx.x * (int64_t)RED_T + threadIdx.x; t < nt; t += (int64_t)gridDim.x * RED_T) {
    double ua[4];
    for (int a = 0; a < 4; ++a) ua[a] = u[tets[a * nt + t]];
    double s = 0.0;
    for (int q = 0; q < QT; ++q) {
      double uq = c_tet_l[q][0] * ua[0] + c_tet_l[q][1] * ua[1] + c_tet_l[q][2] * ua[2] + c_tet_l[q][3] * ua[3];
      double e = exp(uq), ei = 1.0 / e;
      double sh = 0.5 * (e - ei), ch = 0.5 * (e + ei);
      s += c_tet_w[q] * (uq * sh - 2.0 * ch + 2.0);
    }
    acc[0] += vol[t] * s;
  }
  block_reduce_store<1>(acc, part + blockIdx.x);
}

// Values of the sparse operator with J = 0 from the slot descriptors.
__global__ void k_fill_operator(int nnz, const int* __restrict__ kind, const int* __restrict__ ref,
                                const double* __restrict__ a1, const double* __restrict__ a1m, double eps_m,
                                double eps_s,
                                const double* __restrict__ mass_m, const double* __restrict__ corrV_m,
                                const double* __restrict__ corrK_m, const double* __restrict__ mass_s,
                                const double* __restrict__ corrV_s, const double* __restrict__ corrK_s,
                                double* __restrict__ base) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nnz) return;
  int r = ref[s];
  double v = 0.0;
  switch (kind[s]) {
    case 0: v = eps_s * a1[s] + (a1m ? eps_m * a1m[s] : 0.0); break;  // stiffness (Omega_i, Omega_m)
    case 1: v = eps_m * mass_m[r]; break;                      // eps_m R_m' M_m
    case 2: v = -eps_s * mass_s[r]; break;                     // -eps_s R_s' M_s
    case 3: v = 0.5 * mass_m[r] + corrK_m[r]; break;           // (M_m/2 + K_L) near part
    case 4: v = -corrV_m[r]; break;                            // -V_L near part
    case 5: v = 0.5 * mass_s[r] - corrK_s[r]; break;           // (M_s/2 - K_Y) near part
    case 6: v = corrV_s[r]; break;                             // V_Y near part
    case 7: v = 1.0; break;                                    // lam_m rows of Eq. fembem_matrix's
                                                               // solve (Gamma_m interior)
  }
  base[s] = v;
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int launch_tet_volumes(Mesh* m, const int* tets, int64_t nt, double* vol) {
  if (nt == 0) return PBFB_OK;
  k_tet_volumes<<<blocks_for(nt, 256), 256, 0, m->stream>>>(m->xyz.p, m->nv, tets, nt, vol);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_stiffness_local(Mesh* m, const int* tets, int64_t nt, const double* vol, double* loc10) {
  if (nt == 0) return PBFB_OK;
  k_stiffness_local<<<blocks_for(nt, 256), 256, 0, m->stream>>>(m->xyz.p, m->nv, tets, nt, vol, loc10);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_gather(Mesh* m, int nslots, const int* ptr, const int* idx, const double* local, const double* base,
                  double scale, double* out) {
  if (nslots == 0) return PBFB_OK;
  k_gather<<<blocks_for(nslots, 256), 256, 0, m->stream>>>(nslots, ptr, idx, local, base, scale, out);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

// float-float table e^{j/32}, j = -FX_J..FX_J, for exp_pm (once per mesh)
static int fx_table(Mesh* m) {
  if (m->fx_tab.n) return PBFB_OK;
  float2 t[2 * FX_J + 1];
  for (int j = -FX_J; j <= FX_J; ++j) {
    const double v = std::exp(j / 32.0);
    const float h = (float)v;
    t[j + FX_J] = make_float2(h, (float)(v - (double)h));
  }
  return m->fx_tab.upload(t, 2 * FX_J + 1, m->stream);
}

// sinh / cosh on the float32 pipes (exp_pm) in the mixed precision, float64 exp otherwise
static bool use_fx(const Mesh* m) { return m->precision != PBFB_FP64; }

int launch_element_nl(Mesh* m, int scheme, const double* u, double coef, double* loc) {
  cudaEvent_t ev;
  const bool fx = use_fx(m);
  if (fx) PB_TRY(fx_table(m));
  timer_begin(m, m->t_elem, &ev);
  if (fx)
    k_element_nl<true><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(scheme, u, m->tets.p, m->nt, m->vol.p, coef,
                                                                      m->fx_tab.p, loc);
  else
    k_element_nl<false><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(scheme, u, m->tets.p, m->nt, m->vol.p, coef,
                                                                       nullptr, loc);
  PB_LAUNCHED(m);
  timer_end(m, m->t_elem, ev, (double)m->nt);
  return PBFB_OK;
}

int launch_spmv(Mesh* m, const double* x, double* y) {
  cudaEvent_t ev;
  timer_begin(m, m->t_spmv, &ev);
  int n = m->n;
  const int L = m->spmv_lanes > 0 ? m->spmv_lanes : 8;
  const int B = m->spmv_block > 0 ? m->spmv_block : 256;
  const int g = blocks_for((int64_t)n * L, B);
  if (L == 4)
    k_spmv<4><<<g, B, 0, m->stream>>>(n, m->s_ptr.p, m->s_col.p, m->s_val.p, x, y);
  else if (L == 16)
    k_spmv<16><<<g, B, 0, m->stream>>>(n, m->s_ptr.p, m->s_col.p, m->s_val.p, x, y);
  else
    k_spmv<8><<<g, B, 0, m->stream>>>(n, m->s_ptr.p, m->s_col.p, m->s_val.p, x, y);
  PB_LAUNCHED(m);
  timer_end(m, m->t_spmv, ev, (double)m->snnz);
  return PBFB_OK;
}

int launch_csr_spmv(Mesh* m, int nrows, const int* ptr, const int* col, const double* val, const double* x,
                    double* y, bool accumulate) {
  if (nrows == 0) return PBFB_OK;
  k_csr_acc<<<blocks_for((int64_t)nrows * 8, 256), 256, 0, m->stream>>>(nrows, ptr, col, val, x, y,
                                                                        accumulate ? 1 : 0);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_omega_elements(Mesh* m, int scheme, const double* u, const double* du, const double* omegas_dev,
                          int nomega, double coef, double* loc) {
  cudaEvent_t ev;
  const bool fx = use_fx(m);
  if (fx) PB_TRY(fx_table(m));
  timer_begin(m, m->t_elem, &ev);
  if (fx)
    k_omega_elements<true><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(
        scheme, u, du, omegas_dev, nomega, m->tets.p, m->nt, m->vol.p, coef, m->fx_tab.p, loc);
  else
    k_omega_elements<false><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(
        scheme, u, du, omegas_dev, nomega, m->tets.p, m->nt, m->vol.p, coef, nullptr, loc);
  PB_LAUNCHED(m);
  timer_end(m, m->t_elem, ev, (double)m->nt * nomega);
  return PBFB_OK;
}

int launch_omega_dots(Mesh* m, int nomega, const double* loc, const double* c, const double* p, double* dots_dev) {
  int nb = 152;
  dim3 grid(nb, nomega);
  k_omega_dots<<<grid, RED_T, 0, m->stream>>>(m->nv, m->ng_ptr.p, m->ng_idx.p, loc, m->nt, c, p, m->red.p);
  PB_LAUNCHED(m);
  k_sum_partials<<<nomega, 32, 0, m->stream>>>(m->red.p, nb, 7, dots_dev);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_ion_energy(Mesh* m, const double* u, double* out_dev) {
  int nb = 152;
  k_ion_energy<<<nb, RED_T, 0, m->stream>>>(u, m->tets.p, m->nt, m->vol.p, m->red.p);
  PB_LAUNCHED(m);
  k_sum_partials<<<1, 32, 0, m->stream>>>(m->red.p, nb, 1, out_dev);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_fill_operator(Mesh* m) {
  k_fill_operator<<<blocks_for(m->snnz, 256), 256, 0, m->stream>>>(
      m->snnz, m->s_kind.p, m->s_ref.p, m->a1.p, m->full ? m->a1m.p : nullptr, m->eps_m, m->eps_s, m->sm.mass.p, m->sm.corrV.p, m->sm.corrK.p,
      m->ss.mass.p, m->ss.corrV.p, m->ss.corrK.p, m->s_base.p);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

}  // namespace pbfb
