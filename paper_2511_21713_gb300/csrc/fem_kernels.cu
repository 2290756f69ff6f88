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
#include "warp_sum.cuh"

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

// ------------------------------------------------------------ float-float sinh scheme
// The mixed precision evaluates the sinh scheme's element integrals on the float32 pipes
// (GB300's float64 rate is 1/64 of its float32 rate) in float-float arithmetic: a value is a
// pair hi + lo of float32 numbers with |lo| <= ulp(hi) / 2, sums by Knuth's two-sum and products
// by the FMA two-product (Dekker 1971; Ogita, Rump & Oishi 2005), about 2^-47 relative per
// operation.  Only the scaling by eps_s kappa^2 |T| and the conversion of the final sums to
// float64 (in the gather kernels) use the float64 pipes.
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
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return f2_fast(p, e);
}
__device__ __forceinline__ f2 f2_split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double f2_val(f2 a) { return (double)a.h + (double)a.l; }

// Constants as float-float pairs, split at compile time from their float64 values.
#define PBFB_FF(name, x)                                 \
  constexpr float name##_h = (float)(x);                 \
  constexpr float name##_l = (float)((x) - (double)(float)(x))
#define PBFB_FFV(name) (f2{name##_h, name##_l})

// exp = 2^m e^{j/32} e^f: ln 2 = L1 + L2 + L3, L1 with 16 significant bits (m L1 exact for
// |m| <= 128; u_hi - m L1 exact by Sterbenz' lemma), m L2 as an exact FMA two-product.
constexpr float FX_L1 = 0.693145751953125f;
constexpr float FX_L2 = 1.42860682030941723212e-06f;
constexpr float FX_L3 = (float)(0.69314718055994530942 - 0.693145751953125 - (double)FX_L2);
PBFB_FF(FX_SIXTH, 1.0 / 6.0);

// Quadrature orbits of the 14-point tet rule: S31 orbits k = 1, 2 (three barycentrics alpha_k,
// one beta_k, delta_k = beta_k - alpha_k) and the S22 orbit (two c, two d, e = d - c), with
// u_q = alpha_k sum(u) + delta_k u_i and u_P = c sum(u) + e (u_p + u_q) for the pair P = {p, q}.
// The element sums reduce to orbit sums (l_{q,a} l_{q,b} expanded): the products of the weights
// with the orbit parameters below.
PBFB_FF(OR_A1, PBFB_T_A1);
PBFB_FF(OR_D1, PBFB_T_B1 - PBFB_T_A1);
PBFB_FF(OR_A2, PBFB_T_A2);
PBFB_FF(OR_D2, PBFB_T_B2 - PBFB_T_A2);
PBFB_FF(OR_C3, PBFB_T_C3);
PBFB_FF(OR_E3, PBFB_T_D3 - PBFB_T_C3);
PBFB_FF(OR_WA1, PBFB_T_W1 * PBFB_T_A1);
PBFB_FF(OR_WD1, PBFB_T_W1 * (PBFB_T_B1 - PBFB_T_A1));
PBFB_FF(OR_WAA1, PBFB_T_W1 * PBFB_T_A1 * PBFB_T_A1);
PBFB_FF(OR_WAD1, PBFB_T_W1 * PBFB_T_A1 * (PBFB_T_B1 - PBFB_T_A1));
PBFB_FF(OR_WDD1, PBFB_T_W1 * (PBFB_T_B1 - PBFB_T_A1) * (PBFB_T_B1 - PBFB_T_A1));
PBFB_FF(OR_WA2, PBFB_T_W2 * PBFB_T_A2);
PBFB_FF(OR_WD2, PBFB_T_W2 * (PBFB_T_B2 - PBFB_T_A2));
PBFB_FF(OR_WAA2, PBFB_T_W2 * PBFB_T_A2 * PBFB_T_A2);
PBFB_FF(OR_WAD2, PBFB_T_W2 * PBFB_T_A2 * (PBFB_T_B2 - PBFB_T_A2));
PBFB_FF(OR_WDD2, PBFB_T_W2 * (PBFB_T_B2 - PBFB_T_A2) * (PBFB_T_B2 - PBFB_T_A2));
PBFB_FF(OR_WC3, PBFB_T_W3 * PBFB_T_C3);
PBFB_FF(OR_WE3, PBFB_T_W3 * (PBFB_T_D3 - PBFB_T_C3));
PBFB_FF(OR_WCC3, PBFB_T_W3 * PBFB_T_C3 * PBFB_T_C3);
PBFB_FF(OR_WCE3, PBFB_T_W3 * PBFB_T_C3 * (PBFB_T_D3 - PBFB_T_C3));
PBFB_FF(OR_WEE3, PBFB_T_W3 * (PBFB_T_D3 - PBFB_T_C3) * (PBFB_T_D3 - PBFB_T_C3));

constexpr int FX_J = 12;        // tables for j = -FX_J..FX_J
constexpr double FX_UMAX = 60.0;  // float-float path for |u| <= FX_UMAX (e^60 ~ 1.1e26)

// sinh u and cosh u for |u_hi| <= FX_UMAX.  u = m ln2 + j/32 + f with |f| <= 1/64 and
// e^{+-f} = A +- B, A = 1 + f^2/2 + f^4/24 + f^6/720, B = f (1 + f^2/6 + f^4/120 + f^6/5040)
// (truncation below 1e-19).  With v = m ln2 + j/32: sinh u = A sinh v + B cosh v and
// cosh u = A cosh v + B sinh v; sinh v and cosh v come from the float-float table of
// sinh(j/32), cosh(j/32) when m = 0 (so that sinh keeps its relative accuracy near 0) and from
// (2^m e^{j/32} -+ 2^-m e^{-j/32}) / 2 otherwise (|v| > 0.34, no cancellation).
// tab[2 (j + FX_J)] = (e^{j/32}, e^{-j/32}), tab[2 (j + FX_J) + 1] = (sinh(j/32), cosh(j/32)).
__device__ __forceinline__ void ff_sinh_cosh(f2 u, const float4* __restrict__ tab, f2& S, f2& C) {
  const float mf = rintf(__fmul_rn(u.h, 1.44269504088896340736f));
  f2 r = f2_two(__fsub_rn(u.h, __fmul_rn(mf, FX_L1)), u.l);
  const float p2 = __fmul_rn(mf, FX_L2);
  r = f2_add(r, f2{-p2, -__fmaf_rn(mf, FX_L2, -p2)});
  r = f2_add(r, f2{-__fmul_rn(mf, FX_L3), 0.f});
  const float jf = rintf(__fmul_rn(r.h, 32.f));
  const f2 f = f2_two(__fsub_rn(r.h, __fmul_rn(jf, 0.03125f)), r.l);
  const f2 s = f2_mul(f, f);
  const float s2 = __fmul_rn(s.h, s.h);
  const float sa = __fmul_rn(s2, __fmaf_rn(s.h, 1.f / 720.f, 1.f / 24.f));
  const f2 A = f2_add(f2{1.f, 0.f}, f2{__fmul_rn(0.5f, s.h), __fmaf_rn(0.5f, s.l, sa)});
  const float sb = __fmul_rn(s2, __fmaf_rn(s.h, 1.f / 5040.f, 1.f / 120.f));
  const f2 s6 = f2_mul(s, PBFB_FFV(FX_SIXTH));
  const f2 B = f2_mul(f, f2_add(f2{1.f, 0.f}, f2{s6.h, __fadd_rn(s6.l, sb)}));
  const int jt = 2 * ((int)jf + FX_J);
  const float4 te = __ldg(&tab[jt]), th = __ldg(&tab[jt + 1]);
  const int m = (int)mf;
  const float sp = __int_as_float((126 + m) << 23), sm = __int_as_float((126 - m) << 23);  // 2^(m-1), 2^(-m-1)
  const f2 P{__fmul_rn(te.x, sp), __fmul_rn(te.y, sp)}, Q{__fmul_rn(te.z, sm), __fmul_rn(te.w, sm)};
  const bool z = m == 0;
  const f2 sv = z ? f2{th.x, th.y} : f2_add(P, f2_neg(Q));
  const f2 cv = z ? f2{th.z, th.w} : f2_add(P, Q);
  S = f2_add(f2_mul(A, sv), f2_mul(B, cv));
  C = f2_add(f2_mul(A, cv), f2_mul(B, sv));
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

// F, F' and F'' of a scheme in float-float.  The Taylor schemes by Horner's rule on u^2 with the
// ratios of consecutive coefficients (all terms of one sign, no cancellation):
//   F = u (1 + u^2/6 (1 + u^2/20 (1 + u^2/42))), F' = 1 + u^2/2 (1 + u^2/12 (1 + u^2/30)),
// cut at degree 3, 5 or 7; F'' is F one degree lower.  The sinh scheme from ff_sinh_cosh.
PBFB_FF(FX_R6, 1.0 / 6.0);
PBFB_FF(FX_R12, 1.0 / 12.0);
PBFB_FF(FX_R20, 1.0 / 20.0);
PBFB_FF(FX_R30, 1.0 / 30.0);
PBFB_FF(FX_R42, 1.0 / 42.0);

// 1 + u2 r (1 + ...): one Horner step on a float-float tail
__device__ __forceinline__ f2 ff_horner(f2 u2, f2 r, f2 tail) {
  return f2_add(f2{1.f, 0.f}, f2_mul(f2_mul(u2, r), tail));
}

template <int S>
__device__ __forceinline__ void ff_scheme(f2 u, const float4* __restrict__ tab, f2& F, f2& G, f2& H) {
  if (S == PBFB_HS) {
    ff_sinh_cosh(u, tab, F, G);
    H = F;
  } else if (S == PBFB_LINEAR) {
    F = u;
    G = f2{1.f, 0.f};
    H = f2{0.f, 0.f};
  } else {
    const f2 u2 = f2_mul(u, u);
    const f2 one{1.f, 0.f};
    const f2 half_u2{0.5f * u2.h, 0.5f * u2.l};
    // odd part: degree 3 -> u (1 + u2/6); 5 -> u (1 + u2/6 (1 + u2/20)); 7 -> one more factor
    const f2 o7 = S == PBFB_T7 ? ff_horner(u2, PBFB_FFV(FX_R42), one) : one;
    const f2 o5 = S == PBFB_T3 ? one : ff_horner(u2, PBFB_FFV(FX_R20), o7);
    F = f2_mul(u, ff_horner(u2, PBFB_FFV(FX_R6), o5));
    // F'': the odd series one degree lower
    const f2 p5 = S == PBFB_T7 ? ff_horner(u2, PBFB_FFV(FX_R20), one) : one;
    H = S == PBFB_T3 ? u : f2_mul(u, ff_horner(u2, PBFB_FFV(FX_R6), p5));
    // even part: 1 + u2/2 (1 + u2/12 (1 + u2/30)), cut at the scheme's degree - 1
    const f2 e6 = S == PBFB_T7 ? ff_horner(u2, PBFB_FFV(FX_R30), one) : one;
    const f2 e4 = S == PBFB_T3 ? one : ff_horner(u2, PBFB_FFV(FX_R12), e6);
    G = f2_add(one, f2_mul(half_u2, e4));
  }
}

// Jacobian (10 entries, k = 0..9) and load (4 entries) of F on one tet in float64.
__device__ __forceinline__ void element_sums_f64(int scheme, const double (&ua)[4], double (&J)[10],
                                                 double (&N)[4]) {
  for (int k = 0; k < 10; ++k) J[k] = 0.0;
  for (int a = 0; a < 4; ++a) N[a] = 0.0;
  for (int q = 0; q < QT; ++q) {
    double l0 = c_tet_l[q][0], l1 = c_tet_l[q][1], l2 = c_tet_l[q][2], l3 = c_tet_l[q][3];
    double uq = l0 * ua[0] + l1 * ua[1] + l2 * ua[2] + l3 * ua[3];
    double F, Fp, Fpp;
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
}

// The omega batch's three loads of one tet for one omega in float64.
__device__ __forceinline__ void omega_sums_f64(int scheme, const double (&ua)[4], const double (&da)[4], double om,
                                               double (&R0)[4], double (&R1)[4], double (&R2)[4]) {
  for (int a = 0; a < 4; ++a) R0[a] = R1[a] = R2[a] = 0.0;
  for (int q = 0; q < QT; ++q) {
    double l[4] = {c_tet_l[q][0], c_tet_l[q][1], c_tet_l[q][2], c_tet_l[q][3]};
    double uq = l[0] * ua[0] + l[1] * ua[1] + l[2] * ua[2] + l[3] * ua[3];
    double dq = l[0] * da[0] + l[1] * da[1] + l[2] * da[2] + l[3] * da[3];
    double F, Fp, Fpp;
    scheme_F(scheme, uq + om * dq, F, Fp, Fpp);
    double w = c_tet_w[q];
    double f0 = w * F, f1 = w * Fp * dq, f2 = w * Fpp * dq * dq;
    for (int a = 0; a < 4; ++a) {
      R0[a] += f0 * l[a];
      R1[a] += f1 * l[a];
      R2[a] += f2 * l[a];
    }
  }
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

// The same over float-float tet-local entries (the float-float element kernels' output):
// the sum in float-float, one conversion to float64 per slot.
__global__ void k_gather_ff(int nslots, const int* __restrict__ ptr, const int* __restrict__ idx,
                            const float2* __restrict__ local, const double* __restrict__ base, double scale,
                            double* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslots) return;
  f2 acc{0.f, 0.f};
  for (int k = ptr[s]; k < ptr[s + 1]; ++k) {
    const float2 x = local[idx[k]];
    acc = f2_add(acc, f2{x.x, x.y});
  }
  out[s] = (base ? base[s] : 0.0) + scale * f2_val(acc);
}

__device__ __forceinline__ float2 f2_store(f2 a) { return make_float2(a.h, a.l); }

// Jacobian and load of F on one tet (layout k * nt + t: J at k = 0..9, N at k = 10..13).
__global__ void k_element_nl(int scheme, const double* __restrict__ u, const int* __restrict__ tets, int64_t nt,
                             const double* __restrict__ vol, double coef, double* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ua[4];
  for (int a = 0; a < 4; ++a) ua[a] = u[tets[a * nt + t]];
  double J[10], N[4];
  element_sums_f64(scheme, ua, J, N);
  double s = coef * vol[t];
  for (int k = 0; k < 10; ++k) loc[k * nt + t] = s * J[k];
  for (int a = 0; a < 4; ++a) loc[(10 + a) * nt + t] = s * N[a];
}

// Tets outside the float-float range take the float64 sums (kept out of line).
__device__ __noinline__ void element_fallback(int scheme, const double* ua4, double sc, int64_t nt, int64_t t,
                                              float2* __restrict__ loc) {
  const double ua[4] = {ua4[0], ua4[1], ua4[2], ua4[3]};
  double J[10], N[4];
  element_sums_f64(scheme, ua, J, N);
  for (int k = 0; k < 10; ++k) loc[k * nt + t] = f2_store(f2_split(sc * J[k]));
  for (int a = 0; a < 4; ++a) loc[(10 + a) * nt + t] = f2_store(f2_split(sc * N[a]));
}

// Jacobian and load of one tet in float-float (scheme S), from the orbit sums:
//   N_a  = sum_k W_k (alpha_k FS_k + delta_k f_{k,a}) + W_3 (c FS_3 + e sum_{P ∋ a} f_P)
//   J_ab = C + h_a + h_b + [a != b] W_3 e^2 g_{ab},  J_aa = C + 2 h_a + D_a
// with f = F, g = F' at the points, FS / GS the orbit sums, C = sum W alpha^2 GS,
// h_a = sum W alpha delta g_{k,a} (+ W_3 c e sum_{P ∋ a} g_P), D_a = sum W delta^2 g_{k,a}
// (+ W_3 e^2 sum_{P ∋ a} g_P): the 14-point sums of w F l_a and w F' l_a l_b regrouped.
template <int S>
__global__ void __launch_bounds__(128) k_element_ff(const double* __restrict__ u, const int* __restrict__ tets,
                                                    int64_t nt, const double* __restrict__ vol, double coef,
                                                    const float4* __restrict__ tab, float2* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ua[4];
  double umax = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ua[a] = u[tets[a * nt + t]];
    umax = fmax(umax, fabs(ua[a]));
  }
  const double sc = coef * vol[t];
  if (!(umax <= FX_UMAX && fabs(sc) <= 1e10)) {  // |u_q| <= max |u_a| (convex combination)
    element_fallback(S, ua, sc, nt, t, loc);
    return;
  }
  f2 v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = f2_split(ua[a]);
  const f2 su = f2_add(f2_add(v[0], v[1]), f2_add(v[2], v[3]));
  f2 n[4], h[4], D[4], g3[6], T, C;
  {  // S31 orbit 1
    const f2 as = f2_mul(su, PBFB_FFV(OR_A1));
    f2 fs, gs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f2 F, G, H;
      ff_scheme<S>(f2_add(as, f2_mul(v[i], PBFB_FFV(OR_D1))), tab, F, G, H);
      n[i] = f2_mul(F, PBFB_FFV(OR_WD1));
      h[i] = f2_mul(G, PBFB_FFV(OR_WAD1));
      D[i] = f2_mul(G, PBFB_FFV(OR_WDD1));
      fs = i ? f2_add(fs, F) : F;
      gs = i ? f2_add(gs, G) : G;
    }
    T = f2_mul(fs, PBFB_FFV(OR_WA1));
    C = f2_mul(gs, PBFB_FFV(OR_WAA1));
  }
  {  // S31 orbit 2
    const f2 as = f2_mul(su, PBFB_FFV(OR_A2));
    f2 fs, gs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f2 F, G, H;
      ff_scheme<S>(f2_add(as, f2_mul(v[i], PBFB_FFV(OR_D2))), tab, F, G, H);
      n[i] = f2_add(n[i], f2_mul(F, PBFB_FFV(OR_WD2)));
      h[i] = f2_add(h[i], f2_mul(G, PBFB_FFV(OR_WAD2)));
      D[i] = f2_add(D[i], f2_mul(G, PBFB_FFV(OR_WDD2)));
      fs = i ? f2_add(fs, F) : F;
      gs = i ? f2_add(gs, G) : G;
    }
    T = f2_add(T, f2_mul(fs, PBFB_FFV(OR_WA2)));
    C = f2_add(C, f2_mul(gs, PBFB_FFV(OR_WAA2)));
  }
  {  // S22 orbit: pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    const f2 cs = f2_mul(su, PBFB_FFV(OR_C3));
    f2 fs, gs;
#pragma unroll
    for (int p = 0, P = 0; p < 3; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q, ++P) {
        f2 F, G, H;
        ff_scheme<S>(f2_add(cs, f2_mul(f2_add(v[p], v[q]), PBFB_FFV(OR_E3))), tab, F, G, H);
        const f2 fn = f2_mul(F, PBFB_FFV(OR_WE3)), gh = f2_mul(G, PBFB_FFV(OR_WCE3));
        const f2 gd = f2_mul(G, PBFB_FFV(OR_WEE3));
        n[p] = f2_add(n[p], fn);
        n[q] = f2_add(n[q], fn);
        h[p] = f2_add(h[p], gh);
        h[q] = f2_add(h[q], gh);
        D[p] = f2_add(D[p], gd);
        D[q] = f2_add(D[q], gd);
        g3[P] = gd;
        fs = P ? f2_add(fs, F) : F;
        gs = P ? f2_add(gs, G) : G;
      }
    T = f2_add(T, f2_mul(fs, PBFB_FFV(OR_WC3)));
    C = f2_add(C, f2_mul(gs, PBFB_FFV(OR_WCC3)));
  }
  const f2 s = f2_split(sc);
#pragma unroll
  for (int a = 0, P = 0; a < 4; ++a) {
    loc[sym10(a, a) * nt + t] = f2_store(f2_mul(s, f2_add(f2_add(C, D[a]), f2{2.f * h[a].h, 2.f * h[a].l})));
#pragma unroll
    for (int b = a + 1; b < 4; ++b, ++P)
      loc[sym10(a, b) * nt + t] = f2_store(f2_mul(s, f2_add(f2_add(C, g3[P]), f2_add(h[a], h[b]))));
    loc[(10 + a) * nt + t] = f2_store(f2_mul(s, f2_add(T, n[a])));
  }
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
__global__ void k_omega_elements(int scheme, const double* __restrict__ u, const double* __restrict__ du,
                                 const double* __restrict__ omegas, int nomega, const int* __restrict__ tets,
                                 int64_t nt, const double* __restrict__ vol, double coef, double* __restrict__ loc) {
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
    double R0[4], R1[4], R2[4];
    omega_sums_f64(scheme, ua, da, omegas[o], R0, R1, R2);
    int64_t base = (int64_t)o * 12 * nt;
    for (int a = 0; a < 4; ++a) {
      loc[base + (0 * 4 + a) * nt + t] = s * R0[a];
      loc[base + (1 * 4 + a) * nt + t] = s * R1[a];
      loc[base + (2 * 4 + a) * nt + t] = s * R2[a];
    }
  }
}

// Out-of-range omegas of a tet take the float64 loads (kept out of line).
__device__ __noinline__ void omega_fallback(int scheme, const double* ua4, const double* da4, double om, double sc,
                                            int64_t nt, int64_t t, float2* __restrict__ loc) {
  const double ua[4] = {ua4[0], ua4[1], ua4[2], ua4[3]}, da[4] = {da4[0], da4[1], da4[2], da4[3]};
  double R0[4], R1[4], R2[4];
  omega_sums_f64(scheme, ua, da, om, R0, R1, R2);
  for (int a = 0; a < 4; ++a) {
    loc[(0 * 4 + a) * nt + t] = f2_store(f2_split(sc * R0[a]));
    loc[(1 * 4 + a) * nt + t] = f2_store(f2_split(sc * R1[a]));
    loc[(2 * 4 + a) * nt + t] = f2_store(f2_split(sc * R2[a]));
  }
}

// Orbit-sum accumulator of one load sum_q W_q x_q l_{q,a} = T + n_a (see k_element_ff).
struct OrbitLoad {
  f2 T, n[4], s;
};

// Omega batch in float-float (scheme S): per tet and omega the loads of F(w), F'(w) d and
// F''(w) d^2 at w = u + omega du; same layout as k_omega_elements.
template <int S>
__global__ void __launch_bounds__(128) k_omega_ff(const double* __restrict__ u, const double* __restrict__ du,
                                                     const double* __restrict__ omegas, int nomega,
                                                     const int* __restrict__ tets, int64_t nt,
                                                     const double* __restrict__ vol, double coef,
                                                     const float4* __restrict__ tab, float2* __restrict__ loc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ua[4], da[4], dmax = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int vtx = tets[a * nt + t];
    ua[a] = u[vtx];
    da[a] = du[vtx];
    dmax = fmax(dmax, fabs(da[a]));
  }
  const double sc = coef * vol[t];
  const bool scale_ok = fabs(sc) * (1.0 + dmax) * (1.0 + dmax) <= 1e10;
  f2 d[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) d[a] = f2_split(da[a]);
  const f2 sd = f2_add(f2_add(d[0], d[1]), f2_add(d[2], d[3]));
  const f2 s = f2_split(sc);
  for (int o = 0; o < nomega; ++o) {
    const double om = omegas[o];
    float2* out = loc + (int64_t)o * 12 * nt;
    double wmax = 0.0;
    f2 w[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double wa = fma(om, da[a], ua[a]);
      wmax = fmax(wmax, fabs(wa));
      w[a] = f2_split(wa);
    }
    if (!(wmax <= FX_UMAX && scale_ok)) {
      omega_fallback(S, ua, da, om, sc, nt, t, out);
      continue;
    }
    const f2 sw = f2_add(f2_add(w[0], w[1]), f2_add(w[2], w[3]));
    OrbitLoad L[3];
    // one point: x = (F, F' d, F'' d^2); an S31 point adds x W delta to n_i, an S22 point
    // x W e to n_p and n_q; the orbit sums s enter T with W alpha (W c)
    auto point = [&](f2 wq, f2 dq, bool init_n, bool init_s, int i, int j, f2 wn) {
      f2 F, G, H;
      ff_scheme<S>(wq, tab, F, G, H);
      const f2 hd = f2_mul(H, dq);
      const f2 x[3] = {F, f2_mul(G, dq), f2_mul(hd, dq)};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const f2 m = f2_mul(x[k], wn);
        L[k].n[i] = init_n ? m : f2_add(L[k].n[i], m);
        if (j >= 0) L[k].n[j] = f2_add(L[k].n[j], m);
        L[k].s = init_s ? x[k] : f2_add(L[k].s, x[k]);
      }
    };
    {  // S31 orbit 1 (initialises the accumulators)
      const f2 aw = f2_mul(sw, PBFB_FFV(OR_A1)), ad = f2_mul(sd, PBFB_FFV(OR_A1));
#pragma unroll
      for (int i = 0; i < 4; ++i)
        point(f2_add(aw, f2_mul(w[i], PBFB_FFV(OR_D1))), f2_add(ad, f2_mul(d[i], PBFB_FFV(OR_D1))), true, i == 0, i,
              -1, PBFB_FFV(OR_WD1));
#pragma unroll
      for (int k = 0; k < 3; ++k) L[k].T = f2_mul(L[k].s, PBFB_FFV(OR_WA1));
    }
    {  // S31 orbit 2
      const f2 aw = f2_mul(sw, PBFB_FFV(OR_A2)), ad = f2_mul(sd, PBFB_FFV(OR_A2));
#pragma unroll
      for (int i = 0; i < 4; ++i)
        point(f2_add(aw, f2_mul(w[i], PBFB_FFV(OR_D2))), f2_add(ad, f2_mul(d[i], PBFB_FFV(OR_D2))), false, i == 0, i,
              -1, PBFB_FFV(OR_WD2));
#pragma unroll
      for (int k = 0; k < 3; ++k) L[k].T = f2_add(L[k].T, f2_mul(L[k].s, PBFB_FFV(OR_WA2)));
    }
    {  // S22 orbit
      const f2 cw = f2_mul(sw, PBFB_FFV(OR_C3)), cd = f2_mul(sd, PBFB_FFV(OR_C3));
#pragma unroll
      for (int p = 0, P = 0; p < 3; ++p)
#pragma unroll
        for (int q = p + 1; q < 4; ++q, ++P)
          point(f2_add(cw, f2_mul(f2_add(w[p], w[q]), PBFB_FFV(OR_E3))),
                f2_add(cd, f2_mul(f2_add(d[p], d[q]), PBFB_FFV(OR_E3))), false, P == 0, p, q,
                PBFB_FFV(OR_WE3));
#pragma unroll
      for (int k = 0; k < 3; ++k) L[k].T = f2_add(L[k].T, f2_mul(L[k].s, PBFB_FFV(OR_WC3)));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int a = 0; a < 4; ++a) out[(k * 4 + a) * nt + t] = f2_store(f2_mul(s, f2_add(L[k].T, L[k].n[a])));
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
// seven FEM-row dot products; one partial row of 7 per block.  FF: the tet-local entries are
// float-float pairs (summed in float-float, converted once per vertex).
template <bool FF>
__global__ void __launch_bounds__(RED_T) k_omega_dots(int nv, const int* __restrict__ ptr, const int* __restrict__ idx,
                                                      const double* __restrict__ loc, int64_t nt,
                                                      const double* __restrict__ c, const double* __restrict__ p,
                                                      double* __restrict__ part) {
  int o = blockIdx.y;
  const double* L = loc + (int64_t)o * 12 * nt;
  const float2* L2 = reinterpret_cast<const float2*>(L);
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * RED_T + threadIdx.x; i < nv; i += gridDim.x * RED_T) {
    double n0 = 0, n1 = 0, n2 = 0;
    if (FF) {
      f2 a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f};
      for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int e = idx[k];
        const float2 x0 = L2[e], x1 = L2[4 * nt + e], x2 = L2[8 * nt + e];
        a0 = f2_add(a0, f2{x0.x, x0.y});
        a1 = f2_add(a1, f2{x1.x, x1.y});
        a2 = f2_add(a2, f2{x2.x, x2.y});
      }
      n0 = f2_val(a0);
      n1 = f2_val(a1);
      n2 = f2_val(a2);
    } else {
      for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
        int e = idx[k];
        n0 += L[e];
        n1 += L[4 * nt + e];
        n2 += L[8 * nt + e];
      }
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
// (one warp per problem)
__global__ void k_sum_partials(const double* __restrict__ part, int nb, int w, double* __restrict__ out) {
  const int o = blockIdx.x;
  for (int k = 0; k < w; ++k) {
    const double s = warp_strided_sum(part + (int64_t)o * nb * w + k, nb, w);
    if (threadIdx.x == 0) out[o * w + k] = s;
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
                  double scale, double* out, bool ff) {
  if (nslots == 0) return PBFB_OK;
  if (ff)
    k_gather_ff<<<blocks_for(nslots, 256), 256, 0, m->stream>>>(
        nslots, ptr, idx, reinterpret_cast<const float2*>(local), base, scale, out);
  else
    k_gather<<<blocks_for(nslots, 256), 256, 0, m->stream>>>(nslots, ptr, idx, local, base, scale, out);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

// float-float tables of exp(+-j/32) and sinh / cosh(j/32), j = -FX_J..FX_J (once per mesh)
static int fx_table(Mesh* m) {
  if (m->fx_tab.n) return PBFB_OK;
  float4 t[2 * (2 * FX_J + 1)];
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  for (int j = -FX_J; j <= FX_J; ++j) {
    float4 e, c;
    split(std::exp(j / 32.0), e.x, e.y);
    split(std::exp(-j / 32.0), e.z, e.w);
    split(std::sinh(j / 32.0), c.x, c.y);
    split(std::cosh(j / 32.0), c.z, c.w);
    t[2 * (j + FX_J)] = e;
    t[2 * (j + FX_J) + 1] = c;
  }
  return m->fx_tab.upload(t, 2 * (2 * FX_J + 1), m->stream);
}

// The mixed precision runs the element kernels in float-float, the float64 precision in float64.
static bool use_ff(const Mesh* m, int scheme) {
  return m->precision != PBFB_FP64 && scheme >= PBFB_LINEAR && scheme <= PBFB_T7;
}

template <int S>
static void element_ff(Mesh* m, const double* u, double coef, float2* out) {
  k_element_ff<S><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(u, m->tets.p, m->nt, m->vol.p, coef, m->fx_tab.p,
                                                                  out);
}

template <int S>
static void omega_ff(Mesh* m, const double* u, const double* du, const double* omegas, int nomega, double coef,
                     float2* out) {
  k_omega_ff<S><<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(u, du, omegas, nomega, m->tets.p, m->nt, m->vol.p,
                                                                coef, m->fx_tab.p, out);
}

int launch_element_nl(Mesh* m, int scheme, const double* u, double coef, double* loc, bool* ff) {
  cudaEvent_t ev;
  *ff = use_ff(m, scheme);
  if (*ff) PB_TRY(fx_table(m));
  timer_begin(m, m->t_elem, &ev);
  if (*ff) {
    float2* out = reinterpret_cast<float2*>(loc);
    switch (scheme) {
      case PBFB_LINEAR: element_ff<PBFB_LINEAR>(m, u, coef, out); break;
      case PBFB_T3: element_ff<PBFB_T3>(m, u, coef, out); break;
      case PBFB_T5: element_ff<PBFB_T5>(m, u, coef, out); break;
      case PBFB_T7: element_ff<PBFB_T7>(m, u, coef, out); break;
      default: element_ff<PBFB_HS>(m, u, coef, out); break;
    }
  } else
    k_element_nl<<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(scheme, u, m->tets.p, m->nt, m->vol.p, coef, loc);
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
                          int nomega, double coef, double* loc, bool* ff) {
  cudaEvent_t ev;
  *ff = use_ff(m, scheme);
  if (*ff) PB_TRY(fx_table(m));
  timer_begin(m, m->t_elem, &ev);
  if (*ff) {
    float2* out = reinterpret_cast<float2*>(loc);
    switch (scheme) {
      case PBFB_LINEAR: omega_ff<PBFB_LINEAR>(m, u, du, omegas_dev, nomega, coef, out); break;
      case PBFB_T3: omega_ff<PBFB_T3>(m, u, du, omegas_dev, nomega, coef, out); break;
      case PBFB_T5: omega_ff<PBFB_T5>(m, u, du, omegas_dev, nomega, coef, out); break;
      case PBFB_T7: omega_ff<PBFB_T7>(m, u, du, omegas_dev, nomega, coef, out); break;
      default: omega_ff<PBFB_HS>(m, u, du, omegas_dev, nomega, coef, out); break;
    }
  } else
    k_omega_elements<<<blocks_for(m->nt, 128), 128, 0, m->stream>>>(scheme, u, du, omegas_dev, nomega, m->tets.p,
                                                                    m->nt, m->vol.p, coef, loc);
  PB_LAUNCHED(m);
  timer_end(m, m->t_elem, ev, (double)m->nt * nomega);
  return PBFB_OK;
}

int launch_omega_dots(Mesh* m, int nomega, const double* loc, const double* c, const double* p, double* dots_dev,
                      bool ff) {
  int nb = 152;
  dim3 grid(nb, nomega);
  if (ff)
    k_omega_dots<true><<<grid, RED_T, 0, m->stream>>>(m->nv, m->ng_ptr.p, m->ng_idx.p, loc, m->nt, c, p, m->red.p);
  else
    k_omega_dots<false><<<grid, RED_T, 0, m->stream>>>(m->nv, m->ng_ptr.p, m->ng_idx.p, loc, m->nt, c, p, m->red.p);
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
