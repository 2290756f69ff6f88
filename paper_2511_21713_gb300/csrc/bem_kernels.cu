// Boundary-element kernels: Galerkin P1 single- and double-layer operators of the
// Laplace kernel on Gamma_m (Eq. KV) and of the Yukawa kernel on Gamma_s (Sec. 2.2):
//   V_ij = int int psi_i(x) g(x,y) psi_j(y),  K_ij = int int psi_i(x) dg/dn_y(x,y) psi_j(y)
//   g = exp(-kappa r) / (4 pi r),  dg/dn_y = n_y.(x-y) (1 + kappa r) exp(-kappa r) / (4 pi r^3)
// (Laplace is kappa = 0).
//
// Matrix-free far field: every matvec evaluates all pairs of 6-point quadrature
// points of the surface (an N-body sum, coincident points excluded) and reduces the
// target potentials against the test functions.  Touching and close triangle pairs
// are corrected by a precomputed sparse matrix holding, per P1 pair (i, j), the
// difference between the accurate rule of the pair's class and the 6 x 6 rule:
//   identical / common edge / common vertex: Sauter-Schwab (Sauter & Schwab,
//     Boundary Element Methods, 2011, Sec. 5.2), 5 Gauss-Legendre points per variable;
//   near (no shared vertex, centroid distance < 2 max(h_tau, h_sigma)): 6 points on
//     the test triangle x 6 points on each of the 16 sub-triangles of the trial one.
#include <atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "f32x2.cuh"
#include "pbfb_internal.cuh"
#include "quad_tables.cuh"

namespace pbfb {

namespace {

constexpr int NGL = 5;       // Gauss-Legendre points per Sauter-Schwab variable
constexpr int NSUB = 96;     // 16 sub-triangles x 6 points
constexpr double INV4PI = 0.079577471545947667884;

__constant__ double c_gl_x[NGL];
__constant__ double c_gl_w[NGL];
__constant__ double c_sub_b[NSUB][3];
__constant__ double c_sub_w[NSUB];

// Gauss-Legendre nodes on [-1, 1] by Newton's method on the three-term recurrence of
// P_n, mapped to [0, 1].
void gauss_legendre01(int n, double* x01, double* w01) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      pp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      pp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x01[i] = 0.5 * (1.0 - z);
    w01[i] = 1.0 / ((1.0 - z * z) * pp * pp);  // (2 / ((1 - z^2) P'^2)) / 2
  }
}

// ---------------------------------------------------------------- geometry

__global__ void k_surface_geometry(const double* __restrict__ xyz, int nvtot, const int* __restrict__ tri,
                                   const int* __restrict__ vmap, int nt, double cx, double cy, double cz,
                                   double* __restrict__ qx, double* __restrict__ qw, double* __restrict__ nrm,
                                   double* __restrict__ area, float4* __restrict__ qpf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double P[3][3];
  for (int a = 0; a < 3; ++a) {
    int v = vmap[tri[3 * t + a]];
    for (int d = 0; d < 3; ++d) P[a][d] = xyz[d * nvtot + v];
  }
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = P[1][d] - P[0][d];
    e2[d] = P[2][d] - P[0][d];
  }
  double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double nn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  double A = 0.5 * nn;
  area[t] = A;
  for (int d = 0; d < 3; ++d) nrm[d * nt + t] = c[d] / nn;
  int nq = QS * nt;
  for (int q = 0; q < QS; ++q) {
    int j = QS * t + q;
    double y[3];
    for (int d = 0; d < 3; ++d) {
      y[d] = c_tri_b[q][0] * P[0][d] + c_tri_b[q][1] * P[1][d] + c_tri_b[q][2] * P[2][d];
      qx[d * nq + j] = y[d];
    }
    qw[j] = c_tri_w[q] * A;
    qpf[j] = make_float4((float)(y[0] - cx), (float)(y[1] - cy), (float)(y[2] - cz), 0.f);
  }
}

// ---------------------------------------------------------------- near-field corrections

struct PairKer {
  double kappa;
  __device__ __forceinline__ void eval(const double* x, const double* y, const double* n, double& g,
                                       double& dl) const {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    double r = sqrt(r2);
    double e = exp(-kappa * r);
    g = e * INV4PI / r;
    dl = (n[0] * d0 + n[1] * d1 + n[2] * d2) * (1.0 + kappa * r) * e * INV4PI / (r2 * r);
  }
};

// Sauter-Schwab reference points of region `reg` for class `cls` at (xi, e1, e2, e3):
// returns the two points (s1, s2) in {0 <= s2 <= s1 <= 1} and the Jacobian of the map.
__device__ __forceinline__ double ss_point(int cls, int reg, double xi, double e1, double e2, double e3,
                                           double& x1, double& x2, double& y1, double& y2) {
  if (cls == PAIR_IDENTICAL) {
    double a1, a2, b1, b2;
    int base = reg >> 1;
    if (base == 0) {
      a1 = xi; a2 = xi * (1.0 - e1 + e1 * e2);
      b1 = xi * (1.0 - e1 * e2 * e3); b2 = xi * (1.0 - e1);
    } else if (base == 1) {
      a1 = xi; a2 = xi * e1 * (1.0 - e2 + e2 * e3);
      b1 = xi * (1.0 - e1 * e2); b2 = xi * e1 * (1.0 - e2);
    } else {
      a1 = xi * (1.0 - e1 * e2 * e3); a2 = xi * e1 * (1.0 - e2 * e3);
      b1 = xi; b2 = xi * e1 * (1.0 - e2);
    }
    if (reg & 1) { x1 = b1; x2 = b2; y1 = a1; y2 = a2; }
    else { x1 = a1; x2 = a2; y1 = b1; y2 = b2; }
    return xi * xi * xi * e1 * e1 * e2;
  }
  if (cls == PAIR_EDGE) {
    double j = xi * xi * xi * e1 * e1;
    switch (reg) {
      case 0:
        x1 = xi; x2 = xi * e1 * e3; y1 = xi * (1.0 - e1 * e2); y2 = xi * e1 * (1.0 - e2);
        return j;
      case 1:
        x1 = xi; x2 = xi * e1; y1 = xi * (1.0 - e1 * e2 * e3); y2 = xi * e1 * e2 * (1.0 - e3);
        return j * e2;
      case 2:
        x1 = xi * (1.0 - e1 * e2); x2 = xi * e1 * (1.0 - e2); y1 = xi; y2 = xi * e1 * e2 * e3;
        return j * e2;
      case 3:
        x1 = xi * (1.0 - e1 * e2 * e3); x2 = xi * e1 * e2 * (1.0 - e3); y1 = xi; y2 = xi * e1;
        return j * e2;
      default:
        x1 = xi * (1.0 - e1 * e2 * e3); x2 = xi * e1 * (1.0 - e2 * e3); y1 = xi; y2 = xi * e1 * e2;
        return j * e2;
    }
  }
  // common vertex
  if (reg == 0) { x1 = xi; x2 = xi * e1; y1 = xi * e2; y2 = xi * e2 * e3; }
  else { x1 = xi * e2; x2 = xi * e2 * e3; y1 = xi; y2 = xi * e1; }
  return xi * xi * xi * e2;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per special pair.  Outputs, per pair, 9 entries in stored local vertex
// order (a of the test triangle, b of the trial one):
//   corrV/corrK = accurate rule - 6x6 rule (coincident points excluded),
//   fullV = accurate single-layer value (for the operator diagonal),
//   mass = P1 mass entries (identical pairs only).
__global__ void k_pair_corrections(int npair, const int* __restrict__ pt_, const int* __restrict__ ps_,
                                   const int* __restrict__ cls_, const int* __restrict__ perm_,
                                   const int* __restrict__ tri, const int* __restrict__ vmap,
                                   const double* __restrict__ xyz, int nvtot, const double* __restrict__ nrm,
                                   const double* __restrict__ area, const double* __restrict__ qx,
                                   const double* __restrict__ qw, int nt, double kappa,
                                   double* __restrict__ corrV, double* __restrict__ corrK,
                                   double* __restrict__ fullV, double* __restrict__ mass) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= npair) return;
  const int t = pt_[warp], s = ps_[warp], cls = cls_[warp];
  int pt[3], ps[3];
  for (int a = 0; a < 3; ++a) {
    pt[a] = perm_[6 * warp + a];
    ps[a] = perm_[6 * warp + 3 + a];
  }
  double Pt[3][3], Ps[3][3];  // corners in rule order
  for (int a = 0; a < 3; ++a) {
    int vt = vmap[tri[3 * t + pt[a]]], vs = vmap[tri[3 * s + ps[a]]];
    for (int d = 0; d < 3; ++d) {
      Pt[a][d] = xyz[d * nvtot + vt];
      Ps[a][d] = xyz[d * nvtot + vs];
    }
  }
  double ns[3] = {nrm[s], nrm[nt + s], nrm[2 * nt + s]};
  double At = area[t], As = area[s];
  PairKer K{kappa};
  double SL[9], DL[9];
  for (int k = 0; k < 9; ++k) SL[k] = DL[k] = 0.0;
  if (cls != PAIR_NEAR) {
    int nreg = cls == PAIR_IDENTICAL ? 6 : (cls == PAIR_EDGE ? 5 : 2);
    int npts = nreg * NGL * NGL * NGL * NGL;
    for (int k = lane; k < npts; k += 32) {
      int reg = k / (NGL * NGL * NGL * NGL);
      int i = k - reg * (NGL * NGL * NGL * NGL);
      int i0 = i / (NGL * NGL * NGL), i1 = (i / (NGL * NGL)) % NGL, i2 = (i / NGL) % NGL, i3 = i % NGL;
      double x1, x2, y1, y2;
      double jac = ss_point(cls, reg, c_gl_x[i0], c_gl_x[i1], c_gl_x[i2], c_gl_x[i3], x1, x2, y1, y2);
      double W = jac * c_gl_w[i0] * c_gl_w[i1] * c_gl_w[i2] * c_gl_w[i3];
      double bx[3] = {1.0 - x1, x1 - x2, x2}, by[3] = {1.0 - y1, y1 - y2, y2};
      double X[3], Y[3];
      for (int d = 0; d < 3; ++d) {
        X[d] = bx[0] * Pt[0][d] + bx[1] * Pt[1][d] + bx[2] * Pt[2][d];
        Y[d] = by[0] * Ps[0][d] + by[1] * Ps[1][d] + by[2] * Ps[2][d];
      }
      double g, dl;
      K.eval(X, Y, ns, g, dl);
      g *= W;
      dl *= W;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          SL[3 * a + b] += g * bx[a] * by[b];
          DL[3 * a + b] += dl * bx[a] * by[b];
        }
    }
    double jac = 4.0 * At * As;
    for (int k = 0; k < 9; ++k) {
      SL[k] *= jac;
      DL[k] *= jac;
    }
  } else {
    for (int k = lane; k < QS * NSUB; k += 32) {
      int q = k / NSUB, p = k - q * NSUB;
      double X[3], Y[3];
      for (int d = 0; d < 3; ++d) {
        X[d] = c_tri_b[q][0] * Pt[0][d] + c_tri_b[q][1] * Pt[1][d] + c_tri_b[q][2] * Pt[2][d];
        Y[d] = c_sub_b[p][0] * Ps[0][d] + c_sub_b[p][1] * Ps[1][d] + c_sub_b[p][2] * Ps[2][d];
      }
      double g, dl;
      K.eval(X, Y, ns, g, dl);
      double W = c_tri_w[q] * c_sub_w[p] * At * As;
      g *= W;
      dl *= W;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          SL[3 * a + b] += g * c_tri_b[q][a] * c_sub_b[p][b];
          DL[3 * a + b] += dl * c_tri_b[q][a] * c_sub_b[p][b];
        }
    }
  }
  // 6 x 6 rule in stored order (what the far-field sum adds), coincident points excluded
  double RS[9], RD[9];
  for (int k = 0; k < 9; ++k) RS[k] = RD[k] = 0.0;
  int nqt = QS * nt;
  for (int k = lane; k < QS * QS; k += 32) {
    int q = k / QS, p = k - q * QS;
    if (t == s && q == p) continue;
    double X[3], Y[3];
    for (int d = 0; d < 3; ++d) {
      X[d] = qx[d * nqt + QS * t + q];
      Y[d] = qx[d * nqt + QS * s + p];
    }
    double g, dl;
    K.eval(X, Y, ns, g, dl);
    double W = qw[QS * t + q] * qw[QS * s + p];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        RS[3 * a + b] += W * g * c_tri_b[q][a] * c_tri_b[p][b];
        RD[3 * a + b] += W * dl * c_tri_b[q][a] * c_tri_b[p][b];
      }
  }
  for (int k = 0; k < 9; ++k) {
    SL[k] = warp_sum(SL[k]);
    DL[k] = warp_sum(DL[k]);
    RS[k] = warp_sum(RS[k]);
    RD[k] = warp_sum(RD[k]);
  }
  if (lane == 0) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        int o = 9 * warp + 3 * pt[a] + ps[b];  // rule order -> stored order
        int r = 3 * a + b;
        fullV[o] = SL[r];
        corrV[o] = SL[r] - RS[3 * pt[a] + ps[b]];
        corrK[o] = DL[r] - RD[3 * pt[a] + ps[b]];
      }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        mass[9 * warp + 3 * a + b] = (cls == PAIR_IDENTICAL) ? At * (a == b ? 2.0 : 1.0) / 12.0 : 0.0;
  }
}

// ---------------------------------------------------------------- far field

// Source data at every quadrature point j = 6 tau + q:
//   s_j = cs w_j lam_h(y_j)   (single layer),   m_j = cd w_j u_h(y_j) n_tau   (double layer)
__global__ void k_sources(int nt, const int* __restrict__ tri, const int* __restrict__ vmap,
                          const double* __restrict__ lam, const double* __restrict__ u, int u_local,
                          const double* __restrict__ qw, const double* __restrict__ nrm,
                          const float4* __restrict__ qpf, const double* __restrict__ qx, double cs, double cd,
                          int want64, float4* __restrict__ spos, float4* __restrict__ sdl,
                          double* __restrict__ s64) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int nq = QS * nt;
  if (j >= nq) return;
  int t = j / QS, q = j - t * QS;
  double lh = 0.0, uh = 0.0;
  for (int a = 0; a < 3; ++a) {
    int v = tri[3 * t + a];
    double b = c_tri_b[q][a];
    if (lam) lh += b * lam[v];
    if (u) uh += b * u[u_local ? v : vmap[v]];
  }
  double w = qw[j];
  double sv = cs * w * lh, mu = cd * w * uh;
  double n0 = nrm[t], n1 = nrm[nt + t], n2 = nrm[2 * nt + t];
  if (want64) {
    s64[j] = qx[j];
    s64[nq + j] = qx[nq + j];
    s64[2 * nq + j] = qx[2 * nq + j];
    s64[3 * nq + j] = sv;
    s64[4 * nq + j] = mu * n0;
    s64[5 * nq + j] = mu * n1;
    s64[6 * nq + j] = mu * n2;
  } else {
    float4 p = qpf[j];
    p.w = (float)sv;
    spos[j] = p;
    sdl[j] = make_float4((float)(mu * n0), (float)(mu * n1), (float)(mu * n2), 0.f);
  }
}

// float32 N-body: targets = sources = the nq quadrature points.  Block = NT threads, each
// owning TPT targets (interleaved by NT); sources streamed through shared memory in tiles
// of NT; blockIdx.y selects a contiguous source range (split).  Each tile's float partial
// sum is added to a double accumulator.  Coincident points (target index == source
// index) are skipped; only tiles containing one of the thread's targets test for it.
template <int NT, int TPT, bool YUK>
__global__ void __launch_bounds__(NT) k_nbody_f32(int nq, const float4* __restrict__ tgt,
                                                  const float4* __restrict__ spos,
                                                  const float4* __restrict__ sdl, float kappa, int per_split,
                                                  double* __restrict__ out) {
  __shared__ float4 shp[NT];
  __shared__ float4 shd[NT];
  const int t0 = blockIdx.x * NT * TPT;
  int ti[TPT];
  float tx[TPT], ty[TPT], tz[TPT];
  double acc64[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    ti[k] = t0 + k * NT + threadIdx.x;
    float4 p = tgt[ti[k] < nq ? ti[k] : 0];
    tx[k] = p.x;
    ty[k] = p.y;
    tz[k] = p.z;
    acc64[k] = 0.0;
  }
  const int sb = blockIdx.y * per_split;
  const int se = min(nq, sb + per_split);
  const float nk = -kappa * 1.4426950408889634f;  // -kappa log2(e)
  for (int s0 = sb; s0 < se; s0 += NT) {
    int j = s0 + threadIdx.x;
    if (j < se) {
      shp[threadIdx.x] = spos[j];
      shd[threadIdx.x] = sdl[j];
    } else {
      shp[threadIdx.x] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
      shd[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const bool diag = (s0 < t0 + NT * TPT) && (s0 + NT > t0);
    float acc[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) acc[k] = 0.f;
    if (!diag) {
#pragma unroll 4
      for (int jj = 0; jj < NT; ++jj) {
        const float4 p = shp[jj];
        const float4 d = shd[jj];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          float dx = tx[k] - p.x, dy = ty[k] - p.y, dz = tz[k] - p.z;
          float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          float ri = rsqrt_approx(r2);
          float nd = fmaf(d.x, dx, fmaf(d.y, dy, d.z * dz));
          float ri2 = ri * ri;
          if (YUK) {
            float r = r2 * ri;
            float e = ex2_approx(nk * r);
            float kr1 = fmaf(kappa, r, 1.f);
            float tt = fmaf(nd * kr1, ri2, p.w);
            acc[k] = fmaf(tt, e * ri, acc[k]);
          } else {
            float tt = fmaf(nd, ri2, p.w);
            acc[k] = fmaf(tt, ri, acc[k]);
          }
        }
      }
    } else {
      for (int jj = 0; jj < NT; ++jj) {
        const float4 p = shp[jj];
        const float4 d = shd[jj];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          if (s0 + jj == ti[k]) continue;
          float dx = tx[k] - p.x, dy = ty[k] - p.y, dz = tz[k] - p.z;
          float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          float ri = rsqrt_approx(r2);
          float nd = fmaf(d.x, dx, fmaf(d.y, dy, d.z * dz));
          float ri2 = ri * ri;
          if (YUK) {
            float r = r2 * ri;
            float e = ex2_approx(nk * r);
            float kr1 = fmaf(kappa, r, 1.f);
            float tt = fmaf(nd * kr1, ri2, p.w);
            acc[k] = fmaf(tt, e * ri, acc[k]);
          } else {
            float tt = fmaf(nd, ri2, p.w);
            acc[k] = fmaf(tt, ri, acc[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) acc64[k] += (double)acc[k];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k)
    if (ti[k] < nq) out[(int64_t)blockIdx.y * nq + ti[k]] = acc64[k];
}

// Packed variant of k_nbody_f32: two targets per 64-bit register pair, evaluated with the
// Blackwell f32x2 instructions (add/sub/mul/fma on pairs of float32 values), which halve the
// instruction-issue slots of the pair arithmetic; the FP32 lanes do the same work.  Sources are
// staged pre-duplicated ((x,x),(y,y),...) so shared-memory loads give packed operands.  Tiles
// that contain one of the thread's own targets use the scalar path for the coincident-point test.
template <int NT, int NP, bool YUK>
__global__ void __launch_bounds__(NT) k_nbody_f32x2(int nq, const float4* __restrict__ tgt,
                                                    const float4* __restrict__ spos,
                                                    const float4* __restrict__ sdl, float kappa, int per_split,
                                                    double* __restrict__ out) {
  // per source: (x,x),(y,y) | (z,z),(s,s) | (mx,mx),(my,my) | (mz,mz),0
  __shared__ ulonglong2 sh[4][NT];
  __shared__ float4 shp[NT], shd[NT];  // scalar copies for the diagonal tiles
  constexpr int TPT = 2 * NP;
  const int t0 = blockIdx.x * NT * TPT;
  int ti[TPT];
  float txs[TPT], tys[TPT], tzs[TPT];
  f32x2 tx[NP], ty[NP], tz[NP], acc[NP];
  double acc64[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    ti[k] = t0 + k * NT + threadIdx.x;
    float4 p = tgt[ti[k] < nq ? ti[k] : 0];
    txs[k] = p.x;
    tys[k] = p.y;
    tzs[k] = p.z;
    acc64[k] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    tx[k] = pk2(txs[2 * k], txs[2 * k + 1]);
    ty[k] = pk2(tys[2 * k], tys[2 * k + 1]);
    tz[k] = pk2(tzs[2 * k], tzs[2 * k + 1]);
  }
  const int sb = blockIdx.y * per_split;
  const int se = min(nq, sb + per_split);
  const float nk = -kappa * 1.4426950408889634f;
  const f32x2 nk2 = pk2(nk, nk), kap2 = pk2(kappa, kappa), one2 = pk2(1.f, 1.f);
  for (int s0 = sb; s0 < se; s0 += NT) {
    int j = s0 + threadIdx.x;
    float4 p, d;
    if (j < se) {
      p = spos[j];
      d = sdl[j];
    } else {
      p = make_float4(1e18f, 1e18f, 1e18f, 0.f);
      d = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    sh[0][threadIdx.x] = make_ulonglong2(pk2(p.x, p.x), pk2(p.y, p.y));
    sh[1][threadIdx.x] = make_ulonglong2(pk2(p.z, p.z), pk2(p.w, p.w));
    sh[2][threadIdx.x] = make_ulonglong2(pk2(d.x, d.x), pk2(d.y, d.y));
    sh[3][threadIdx.x] = make_ulonglong2(pk2(d.z, d.z), 0ull);
    shp[threadIdx.x] = p;
    shd[threadIdx.x] = d;
    __syncthreads();
    const bool diag = (s0 < t0 + NT * TPT) && (s0 + NT > t0);
    if (!diag) {
#pragma unroll
      for (int k = 0; k < NP; ++k) acc[k] = 0ull;
#pragma unroll 2
      for (int jj = 0; jj < NT; ++jj) {
        const ulonglong2 a0 = sh[0][jj], a1 = sh[1][jj], a2 = sh[2][jj], a3 = sh[3][jj];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          f32x2 dx = sub2(tx[k], a0.x), dy = sub2(ty[k], a0.y), dz = sub2(tz[k], a1.x);
          f32x2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
          float ra, rb;
          upk2(r2, ra, rb);
          f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
          f32x2 nd = fma2(a3.x, dz, fma2(a2.y, dy, mul2(a2.x, dx)));
          f32x2 ri2 = mul2(ri, ri);
          if (YUK) {
            f32x2 r = mul2(r2, ri);
            float xa, xb;
            upk2(mul2(nk2, r), xa, xb);
            f32x2 e = pk2(ex2_approx(xa), ex2_approx(xb));
            f32x2 tt = fma2(mul2(nd, fma2(kap2, r, one2)), ri2, a1.y);
            acc[k] = fma2(tt, mul2(e, ri), acc[k]);
          } else {
            acc[k] = fma2(fma2(nd, ri2, a1.y), ri, acc[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float a, b;
        upk2(acc[k], a, b);
        acc64[2 * k] += (double)a;
        acc64[2 * k + 1] += (double)b;
      }
    } else {
      float accs[TPT];
#pragma unroll
      for (int k = 0; k < TPT; ++k) accs[k] = 0.f;
      for (int jj = 0; jj < NT; ++jj) {
        const float4 p = shp[jj];
        const float4 d = shd[jj];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          if (s0 + jj == ti[k]) continue;
          float dx = txs[k] - p.x, dy = tys[k] - p.y, dz = tzs[k] - p.z;
          float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          float ri = rsqrt_approx(r2);
          float nd = fmaf(d.x, dx, fmaf(d.y, dy, d.z * dz));
          float ri2 = ri * ri;
          if (YUK) {
            float r = r2 * ri;
            float e = ex2_approx(nk * r);
            float kr1 = fmaf(kappa, r, 1.f);
            float tt = fmaf(nd * kr1, ri2, p.w);
            accs[k] = fmaf(tt, e * ri, accs[k]);
          } else {
            float tt = fmaf(nd, ri2, p.w);
            accs[k] = fmaf(tt, ri, accs[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < TPT; ++k) acc64[k] += (double)accs[k];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k)
    if (ti[k] < nq) out[(int64_t)blockIdx.y * nq + ti[k]] = acc64[k];
}

// Mutual float32 N-body for the GMRES operator: every unordered pair of points evaluated once
// for both directions (the organisation of k_nbody_ffm, with one-warp blocks).  Block (rg, cg)
// is one warp; it holds 4 targets per lane (I * 128 + lane + 32 k) as two f32x2 pairs, streams
// the 128 points of tile J through shared memory, and at step s lane l takes point (l + s) mod
// 128, so the 32 lanes update distinct source-side sums (warp-synchronous, fixed order).  Pair
// (i, j): d = x_i - x_j, f = (1 + kappa r) / r^2, g = exp(-kappa r) / r;
//   to i: (s_j + (m_j . d) f) g,   to j: (s_i - (m_i . d) f) g.
constexpr int FM_T = 128;

template <bool YUK>
__global__ void __launch_bounds__(32) k_nbody_f32m(int nq, int G, const float4* __restrict__ spos,
                                                   const float4* __restrict__ sdl, float kappa,
                                                   double* __restrict__ PI, double* __restrict__ PJ) {
  __shared__ float4 sp[FM_T], sd[FM_T];
  __shared__ float accj[FM_T];
  int t = blockIdx.x, rg = 0;
  while (t >= G - rg) {
    t -= G - rg;
    ++rg;
  }
  const int cg = rg + t;
  const int nT = (nq + FM_T - 1) / FM_T;
  const int tpg = (nT + G - 1) / G;
  const int i0g = rg * tpg, i1g = min(nT, (rg + 1) * tpg);
  const int j0g = cg * tpg, j1g = min(nT, (cg + 1) * tpg);
  const int lane = threadIdx.x;
  const float nk = -kappa * 1.4426950408889634f;
  const f32x2 nk2 = pk2(nk, nk), kap2 = pk2(kappa, kappa), one2 = pk2(1.f, 1.f);
  for (int I = i0g; I < i1g; ++I) {
    float tx[4], ty[4], tz[4], ts[4], tmx[4], tmy[4], tmz[4];
    int ti[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ti[k] = I * FM_T + lane + 32 * k;
      const bool v = ti[k] < nq;
      const float4 p = v ? spos[ti[k]] : make_float4(2e15f, 0.f, 0.f, 0.f);
      const float4 d = v ? sdl[ti[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
      tx[k] = p.x;
      ty[k] = p.y;
      tz[k] = p.z;
      ts[k] = p.w;
      tmx[k] = -d.x;  // negated: the source-side term needs -(m_i . d)
      tmy[k] = -d.y;
      tmz[k] = -d.z;
    }
    f32x2 TX[2], TY[2], TZ[2], TS[2], NMX[2], NMY[2], NMZ[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      TX[c] = pk2(tx[2 * c], tx[2 * c + 1]);
      TY[c] = pk2(ty[2 * c], ty[2 * c + 1]);
      TZ[c] = pk2(tz[2 * c], tz[2 * c + 1]);
      TS[c] = pk2(ts[2 * c], ts[2 * c + 1]);
      NMX[c] = pk2(tmx[2 * c], tmx[2 * c + 1]);
      NMY[c] = pk2(tmy[2 * c], tmy[2 * c + 1]);
      NMZ[c] = pk2(tmz[2 * c], tmz[2 * c + 1]);
    }
    double acc64[4] = {0.0, 0.0, 0.0, 0.0};
    for (int J = max(I, j0g); J < j1g; ++J) {
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int jl = J * FM_T + lane + 32 * k;
        if (jl < nq) {
          sp[lane + 32 * k] = spos[jl];
          sd[lane + 32 * k] = sdl[jl];
        } else {
          sp[lane + 32 * k] = make_float4(1e15f, 0.f, 0.f, 0.f);
          sd[lane + 32 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        accj[lane + 32 * k] = 0.f;
      }
      __syncwarp();
      const int cnt = min(FM_T, nq - J * FM_T);
      if (J == I) {
        // diagonal tile: target side only, coincident point skipped
        float a[4] = {0.f, 0.f, 0.f, 0.f};
        for (int jj = 0; jj < cnt; ++jj) {
          const float4 p = sp[jj], d = sd[jj];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (jj == lane + 32 * k) continue;
            const float dx = tx[k] - p.x, dy = ty[k] - p.y, dz = tz[k] - p.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_approx(r2);
            const float nd = fmaf(d.x, dx, fmaf(d.y, dy, d.z * dz));
            const float ri2 = ri * ri;
            if (YUK) {
              const float r = r2 * ri;
              const float e = ex2_approx(nk * r);
              const float tt = fmaf(nd * fmaf(kappa, r, 1.f), ri2, p.w);
              a[k] = fmaf(tt, e * ri, a[k]);
            } else {
              a[k] = fmaf(fmaf(nd, ri2, p.w), ri, a[k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc64[k] += (double)a[k];
      } else {
        f32x2 acc[2] = {0ull, 0ull};
#pragma unroll 2
        for (int st = 0; st < FM_T; ++st) {
          const int jj = (lane + st) & (FM_T - 1);
          const float4 p = sp[jj], d = sd[jj];
          const f32x2 PX = pk2(p.x, p.x), PY = pk2(p.y, p.y), PZ = pk2(p.z, p.z), PS = pk2(p.w, p.w);
          const f32x2 MX = pk2(d.x, d.x), MY = pk2(d.y, d.y), MZ = pk2(d.z, d.z);
          float cj = 0.f;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const f32x2 dx = sub2(TX[c], PX), dy = sub2(TY[c], PY), dz = sub2(TZ[c], PZ);
            const f32x2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            float ra, rb;
            upk2(r2, ra, rb);
            const f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
            const f32x2 ri2 = mul2(ri, ri);
            f32x2 f, g;
            if (YUK) {
              const f32x2 r = mul2(r2, ri);
              float xa, xb;
              upk2(mul2(nk2, r), xa, xb);
              const f32x2 e = pk2(ex2_approx(xa), ex2_approx(xb));
              f = mul2(fma2(kap2, r, one2), ri2);
              g = mul2(e, ri);
            } else {
              f = ri2;
              g = ri;
            }
            const f32x2 ndj = fma2(MZ, dz, fma2(MY, dy, mul2(MX, dx)));
            acc[c] = fma2(fma2(ndj, f, PS), g, acc[c]);
            const f32x2 ndi = fma2(NMZ[c], dz, fma2(NMY[c], dy, mul2(NMX[c], dx)));
            float u0, u1;
            upk2(mul2(fma2(ndi, f, TS[c]), g), u0, u1);
            cj += u0 + u1;
          }
          accj[jj] += cj;
          __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float a0, a1;
          upk2(acc[c], a0, a1);
          acc64[2 * c] += (double)a0;
          acc64[2 * c + 1] += (double)a1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int jl = J * FM_T + lane + 32 * k;
          if (jl < nq) PJ[(int64_t)rg * nq + jl] += (double)accj[lane + 32 * k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (ti[k] < nq) PI[(int64_t)cg * nq + ti[k]] = acc64[k];
  }
}

// float64 N-body, same organisation (one target per thread).
template <int NT, bool YUK>
__global__ void __launch_bounds__(NT) k_nbody_f64(int nq, const double* __restrict__ s64, double kappa,
                                                  int per_split, double* __restrict__ out) {
  __shared__ double sh[7][NT];
  const int i = blockIdx.x * NT + threadIdx.x;
  const int ii = i < nq ? i : 0;
  const double x = s64[ii], y = s64[nq + ii], z = s64[2 * nq + ii];
  const int sb = blockIdx.y * per_split;
  const int se = min(nq, sb + per_split);
  double acc = 0.0;
  for (int s0 = sb; s0 < se; s0 += NT) {
    int j = s0 + threadIdx.x;
    if (j < se) {
      for (int c = 0; c < 7; ++c) sh[c][threadIdx.x] = s64[c * nq + j];
    } else {
      sh[0][threadIdx.x] = sh[1][threadIdx.x] = sh[2][threadIdx.x] = 1e150;
      for (int c = 3; c < 7; ++c) sh[c][threadIdx.x] = 0.0;
    }
    __syncthreads();
    const int cnt = min(NT, se - s0);
    for (int jj = 0; jj < cnt; ++jj) {
      if (s0 + jj == i) continue;
      double dx = x - sh[0][jj], dy = y - sh[1][jj], dz = z - sh[2][jj];
      double r2 = dx * dx + dy * dy + dz * dz;
      double ri = rsqrt(r2);
      double nd = sh[4][jj] * dx + sh[5][jj] * dy + sh[6][jj] * dz;
      double ri2 = ri * ri;
      if (YUK) {
        double r = r2 * ri;
        double e = exp(-kappa * r);
        acc += (sh[3][jj] + nd * (1.0 + kappa * r) * ri2) * e * ri;
      } else {
        acc += (sh[3][jj] + nd * ri2) * ri;
      }
    }
    __syncthreads();
  }
  if (i < nq) out[(int64_t)blockIdx.y * nq + i] = acc;
}

// ---------------------------------------------------------------- float-float far field
//
// The Newton residual needs a far field accurate to float64 level, but the float64 rate of
// GB300 is 1/64 of its float32 rate.  These kernels evaluate the same pair sums in
// float-float arithmetic: every quantity is an unevaluated pair hi + lo of float32 values
// (about 48 significant bits), built from error-free transformations -- Knuth's TwoSum,
// Dekker's FastTwoSum (|a| >= |b|) and the FMA TwoProduct -- as in Ogita, Rump & Oishi,
// "Accurate sum and dot product" (SIAM J. Sci. Comput. 2005).  1/sqrt uses one Newton step
// from the hardware estimate; exp(-x) for the Yukawa kernel uses two float-float tables of
// exp(-k delta) (delta = 1/256) and a 5-term Taylor series for the remainder f < delta.
// The _rn intrinsics keep the compiler from contracting the transformations into FMAs.

constexpr int FF_TABLE_HI = 640;      // exp(-16 delta k1), k1 < 640: x up to 40
constexpr float FF_XMAX = 39.99f;      // exp(-40) ~ 4e-18: larger arguments give 0

__constant__ float2 c_ff_exp_lo[16];   // exp(-delta k0), k0 < 16

struct ff { float h, l; };

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  float lo = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sq(ff a) {
  float p = __fmul_rn(a.h, a.h);
  float e = __fmaf_rn(a.h, a.h, -p);
  e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
  return fast_two_sum(p, e);
}
// difference of two float-float coordinates whose high parts lie on a common grid q, fine enough
// that xh - yh is exact: (xh - yh) + (xl - yl) with |xl - yl| <= q <= |xh - yh| unless xh = yh,
// so a FastTwoSum renormalises it
__device__ __forceinline__ ff ff_diff(float xh, float xl, float yh, float yl) {
  return fast_two_sum(__fsub_rn(xh, yh), __fsub_rn(xl, yl));
}
// a.x + b.y + c.z for float-float vectors
__device__ __forceinline__ ff ff_dot3(ff a0, ff a1, ff a2, ff b0, ff b1, ff b2) {
  float p0 = __fmul_rn(a0.h, b0.h), p1 = __fmul_rn(a1.h, b1.h), p2 = __fmul_rn(a2.h, b2.h);
  float e0 = __fmaf_rn(a0.l, b0.h, __fmaf_rn(a0.h, b0.l, __fmaf_rn(a0.h, b0.h, -p0)));
  float e1 = __fmaf_rn(a1.l, b1.h, __fmaf_rn(a1.h, b1.l, __fmaf_rn(a1.h, b1.h, -p1)));
  float e2 = __fmaf_rn(a2.l, b2.h, __fmaf_rn(a2.h, b2.l, __fmaf_rn(a2.h, b2.h, -p2)));
  ff s1 = two_sum(p0, p1);
  ff s2 = two_sum(s1.h, p2);
  float lo = __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(e0, e1), e2));
  return fast_two_sum(s2.h, lo);
}
// 1/sqrt(r) for r = rh + rl > 0: one Newton step y0 (1 - (r y0^2 - 1)/2) from the hardware estimate
__device__ __forceinline__ ff ff_rsqrt(ff r) {
  float y0 = rsqrtf(r.h);
  float t = __fmul_rn(y0, y0);
  float te = __fmaf_rn(y0, y0, -t);
  float a = __fmul_rn(r.h, t);
  float ae = __fmaf_rn(r.h, t, -a);
  float z = __fadd_rn(__fsub_rn(a, 1.0f), __fmaf_rn(r.l, t, __fmaf_rn(r.h, te, ae)));
  return fast_two_sum(y0, __fmul_rn(__fmul_rn(-0.5f, y0), z));
}
// exp(-x), 0 <= x (float-float); tab_hi in shared memory: exp(-16 k1 / 256)
__device__ __forceinline__ ff ff_expm(ff x, const float2* __restrict__ tab_hi) {
  if (x.h >= FF_XMAX) return {0.f, 0.f};
  int k = __float2int_rd(__fmul_rn(x.h, 256.0f));
  k = k < 0 ? 0 : k;
  ff f = fast_two_sum(__fsub_rn(x.h, __fmul_rn((float)k, 0.00390625f)), x.l);   // 0 <= f < 1/256 (+rounding)
  // exp(-f) = (1 - f) + f^2/2 + f^2 (-f/6 + f^2/24 - f^3/120)
  ff f2 = ff_sq(f);
  float p2 = __fmul_rn(f.h, __fmaf_rn(f.h, __fmaf_rn(f.h, -1.0f / 120.0f, 1.0f / 24.0f), -1.0f / 6.0f));
  ff one_minus = two_sum(1.0f, -f.h);
  one_minus = fast_two_sum(one_minus.h, __fsub_rn(one_minus.l, f.l));
  ff tail = fast_two_sum(__fmul_rn(0.5f, f2.h), __fmaf_rn(f2.h, p2, __fmul_rn(0.5f, f2.l)));
  ff ef = ff_add(one_minus, tail);
  float2 a = tab_hi[k >> 4];
  float2 b = c_ff_exp_lo[k & 15];
  return ff_mul(ff_mul(ef, ff{a.x, a.y}), ff{b.x, b.y});
}

// Float-float sources: 4 float4 per point: (y hi, s hi), (y lo, s lo), (m hi, 0), (m lo, 0),
// with y relative to the surface centre, s = cs w lam_h, m = cd w u_h n.  The coordinates' high
// parts lie on `grid` (a power of 2) with every difference of two of them exact in float32,
// the low parts are the remainders (|y lo| <= grid / 2).
__global__ void k_sources_ff(int nt, const int* __restrict__ tri, const int* __restrict__ vmap,
                             const double* __restrict__ lam, const double* __restrict__ u, int u_local,
                             const double* __restrict__ qw, const double* __restrict__ nrm,
                             const double* __restrict__ qx, double cx, double cy, double cz, double cs, double cd,
                             double grid, float4* __restrict__ src, float4* __restrict__ tgt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int nq = QS * nt;
  if (j >= nq) return;
  int t = j / QS, q = j - t * QS;
  double lh = 0.0, uh = 0.0;
  for (int a = 0; a < 3; ++a) {
    int v = tri[3 * t + a];
    double b = c_tri_b[q][a];
    if (lam) lh += b * lam[v];
    if (u) uh += b * u[u_local ? v : vmap[v]];
  }
  double w = qw[j];
  double sv = cs * w * lh, mu = cd * w * uh;
  double y[3] = {qx[j] - cx, qx[nq + j] - cy, qx[2 * nq + j] - cz};
  double mm[3] = {mu * nrm[t], mu * nrm[nt + t], mu * nrm[2 * nt + t]};
  float yh[3], yl[3], mh[3], ml[3];
  for (int d = 0; d < 3; ++d) {
    const double yq = rint(y[d] / grid) * grid;  // on the grid: exact in float32
    yh[d] = (float)yq;
    yl[d] = (float)(y[d] - yq);
    mh[d] = (float)mm[d];
    ml[d] = (float)(mm[d] - (double)mh[d]);
  }
  float sh = (float)sv, sl = (float)(sv - (double)sh);
  src[4 * j + 0] = make_float4(yh[0], yh[1], yh[2], sh);
  src[4 * j + 1] = make_float4(yl[0], yl[1], yl[2], sl);
  src[4 * j + 2] = make_float4(mh[0], mh[1], mh[2], 0.f);
  src[4 * j + 3] = make_float4(ml[0], ml[1], ml[2], 0.f);
  tgt[2 * j + 0] = make_float4(yh[0], yh[1], yh[2], 0.f);
  tgt[2 * j + 1] = make_float4(yl[0], yl[1], yl[2], 0.f);
}

// One pair in float-float: (s + nd (1 + kappa r) / r^2) exp(-kappa r) / r  (kappa = 0: Laplace)
template <bool YUK>
__device__ __forceinline__ ff ff_pair(const float4& ph, const float4& pl, const float4& mh, const float4& ml,
                                      const float (&th)[3], const float (&tl)[3], ff kap,
                                      const float2* __restrict__ tab) {
  ff d0 = ff_diff(th[0], tl[0], ph.x, pl.x);
  ff d1 = ff_diff(th[1], tl[1], ph.y, pl.y);
  ff d2 = ff_diff(th[2], tl[2], ph.z, pl.z);
  ff r2 = ff_dot3(d0, d1, d2, d0, d1, d2);
  ff ri = ff_rsqrt(r2);
  ff nd = ff_dot3(ff{mh.x, ml.x}, ff{mh.y, ml.y}, ff{mh.z, ml.z}, d0, d1, d2);
  ff ri2 = ff_sq(ri);
  if (YUK) {
    ff r = ff_mul(r2, ri);
    ff x = ff_mul(kap, r);
    ff e = ff_expm(x, tab);
    ff one_x = two_sum(1.0f, x.h);
    one_x = fast_two_sum(one_x.h, __fadd_rn(one_x.l, x.l));
    ff t = ff_add(ff{ph.w, pl.w}, ff_mul(ff_mul(nd, one_x), ri2));
    return ff_mul(t, ff_mul(e, ri));
  }
  ff t = ff_add(ff{ph.w, pl.w}, ff_mul(nd, ri2));
  return ff_mul(t, ri);
}

// Float-float N-body: same tiling as the float32 kernel (one target per thread); each tile's
// float-float partial sum is added to a float64 accumulator.
template <int NT, bool YUK>
__global__ void __launch_bounds__(NT) k_nbody_ff(int nq, const float4* __restrict__ tgt,
                                                 const float4* __restrict__ src, float kh, float kl,
                                                 const float2* __restrict__ tab_hi, int per_split,
                                                 double* __restrict__ out) {
  __shared__ float4 sh[4][NT];
  __shared__ float2 tab[YUK ? FF_TABLE_HI : 1];
  if (YUK)
    for (int k = threadIdx.x; k < FF_TABLE_HI; k += NT) tab[k] = tab_hi[k];
  const int i = blockIdx.x * NT + threadIdx.x;
  const int ii = i < nq ? i : 0;
  const float4 a = tgt[2 * ii], b = tgt[2 * ii + 1];
  const float th[3] = {a.x, a.y, a.z}, tl[3] = {b.x, b.y, b.z};
  const ff kap{kh, kl};
  const int sb = blockIdx.y * per_split;
  const int se = min(nq, sb + per_split);
  double acc64 = 0.0;
  for (int s0 = sb; s0 < se; s0 += NT) {
    int j = s0 + threadIdx.x;
    if (j < se) {
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = src[4 * j + c];
    }
    __syncthreads();
    const int cnt = min(NT, se - s0);
    ff acc{0.f, 0.f};
    for (int jj = 0; jj < cnt; ++jj) {
      if (s0 + jj == i) continue;
      ff v = ff_pair<YUK>(sh[0][jj], sh[1][jj], sh[2][jj], sh[3][jj], th, tl, kap, tab);
      acc = ff_add(acc, v);
    }
    acc64 += (double)acc.h + (double)acc.l;
    __syncthreads();
  }
  if (i < nq) out[(int64_t)blockIdx.y * nq + i] = acc64;
}

// Packed float-float N-body: two targets per thread, every float-float operation applied to both
// with the Blackwell float2 arithmetic (__fadd2_rn / __fmul2_rn / __ffma2_rn, per component the
// same rounding as the scalar _rn operations), halving the issue slots of k_nbody_ff.  Each lane
// performs the scalar kernel's operation sequence under the same source split (results agree to
// float-float rounding).  Sources are staged pre-duplicated; tiles holding one of the thread's
// own targets take the scalar path for the coincident-point test.
struct ffv { float2 h, l; };
__device__ __forceinline__ float2 vdup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ ffv v_two_sum(float2 a, float2 b) {
  float2 s = vadd(a, b);
  float2 bb = vsub(s, a);
  float2 e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
  return {s, e};
}
__device__ __forceinline__ ffv v_fast_two_sum(float2 a, float2 b) {
  float2 s = vadd(a, b);
  return {s, vsub(b, vsub(s, a))};
}
__device__ __forceinline__ ffv v_add(ffv a, ffv b) {
  ffv s = v_two_sum(a.h, b.h);
  float2 lo = vadd(s.l, vadd(a.l, b.l));
  return v_fast_two_sum(s.h, lo);
}
__device__ __forceinline__ ffv v_mul(ffv a, ffv b) {
  float2 p = vmul(a.h, b.h);
  float2 e = vfma(a.h, b.h, vneg(p));
  e = vfma(a.h, b.l, e);
  e = vfma(a.l, b.h, e);
  return v_fast_two_sum(p, e);
}
__device__ __forceinline__ ffv v_sq(ffv a) {
  float2 p = vmul(a.h, a.h);
  float2 e = vfma(a.h, a.h, vneg(p));
  e = vfma(vadd(a.h, a.h), a.l, e);
  return v_fast_two_sum(p, e);
}
__device__ __forceinline__ ffv v_diff(float2 xh, float2 xl, float2 yh, float2 yl) {
  return v_fast_two_sum(vsub(xh, yh), vsub(xl, yl));
}
__device__ __forceinline__ ffv v_dot3(ffv a0, ffv a1, ffv a2, ffv b0, ffv b1, ffv b2) {
  float2 p0 = vmul(a0.h, b0.h), p1 = vmul(a1.h, b1.h), p2 = vmul(a2.h, b2.h);
  float2 e0 = vfma(a0.l, b0.h, vfma(a0.h, b0.l, vfma(a0.h, b0.h, vneg(p0))));
  float2 e1 = vfma(a1.l, b1.h, vfma(a1.h, b1.l, vfma(a1.h, b1.h, vneg(p1))));
  float2 e2 = vfma(a2.l, b2.h, vfma(a2.h, b2.l, vfma(a2.h, b2.h, vneg(p2))));
  ffv s1 = v_two_sum(p0, p1);
  ffv s2 = v_two_sum(s1.h, p2);
  float2 lo = vadd(vadd(s1.l, s2.l), vadd(vadd(e0, e1), e2));
  return v_fast_two_sum(s2.h, lo);
}
__device__ __forceinline__ ffv v_rsqrt(ffv r) {
  float2 y0 = make_float2(rsqrtf(r.h.x), rsqrtf(r.h.y));
  float2 t = vmul(y0, y0);
  float2 te = vfma(y0, y0, vneg(t));
  float2 a = vmul(r.h, t);
  float2 ae = vfma(r.h, t, vneg(a));
  float2 z = vadd(vsub(a, vdup(1.0f)), vfma(r.l, t, vfma(r.h, te, ae)));
  return v_fast_two_sum(y0, vmul(vmul(vdup(-0.5f), y0), z));
}
// exp(-x) per lane as ff_expm; the table index is clamped and the lanes with x >= FF_XMAX give 0
__device__ __forceinline__ ffv v_expm(ffv x, const float2* __restrict__ tab_hi) {
  float2 xs = vmul(x.h, vdup(256.0f));
  int k0 = __float2int_rd(xs.x), k1 = __float2int_rd(xs.y);
  k0 = min(max(k0, 0), FF_TABLE_HI * 16 - 1);
  k1 = min(max(k1, 0), FF_TABLE_HI * 16 - 1);
  float2 kf = vmul(make_float2((float)k0, (float)k1), vdup(0.00390625f));
  ffv f = v_fast_two_sum(vsub(x.h, kf), x.l);
  ffv f2 = v_sq(f);
  float2 p2 = vmul(f.h, vfma(f.h, vfma(f.h, vdup(-1.0f / 120.0f), vdup(1.0f / 24.0f)), vdup(-1.0f / 6.0f)));
  ffv one_minus = v_two_sum(vdup(1.0f), vneg(f.h));
  one_minus = v_fast_two_sum(one_minus.h, vsub(one_minus.l, f.l));
  ffv tail = v_fast_two_sum(vmul(vdup(0.5f), f2.h), vfma(f2.h, p2, vmul(vdup(0.5f), f2.l)));
  ffv ef = v_add(one_minus, tail);
  const float2 a0 = tab_hi[k0 >> 4], a1 = tab_hi[k1 >> 4];
  const float2 b0 = c_ff_exp_lo[k0 & 15], b1 = c_ff_exp_lo[k1 & 15];
  ffv r = v_mul(v_mul(ef, ffv{make_float2(a0.x, a1.x), make_float2(a0.y, a1.y)}),
                ffv{make_float2(b0.x, b1.x), make_float2(b0.y, b1.y)});
  if (x.h.x >= FF_XMAX) r.h.x = r.l.x = 0.f;
  if (x.h.y >= FF_XMAX) r.h.y = r.l.y = 0.f;
  return r;
}

// per source, duplicated: yh.x yh.y | yh.z sh | yl.x yl.y | yl.z sl | mh.x mh.y | mh.z ml.x | ml.y ml.z
template <bool YUK>
__device__ __forceinline__ ffv v_pair(const float4* __restrict__ q, const float2 (&th)[3], const float2 (&tl)[3],
                                      ffv kap, const float2* __restrict__ tab) {
  const float4 c0 = q[0], c1 = q[1], c2 = q[2], c3 = q[3], c4 = q[4], c5 = q[5], c6 = q[6];
  const float2 pxh = make_float2(c0.x, c0.y), pyh = make_float2(c0.z, c0.w);
  const float2 pzh = make_float2(c1.x, c1.y), sh = make_float2(c1.z, c1.w);
  const float2 pxl = make_float2(c2.x, c2.y), pyl = make_float2(c2.z, c2.w);
  const float2 pzl = make_float2(c3.x, c3.y), sl = make_float2(c3.z, c3.w);
  const ffv mx{make_float2(c4.x, c4.y), make_float2(c5.z, c5.w)};
  const ffv my{make_float2(c4.z, c4.w), make_float2(c6.x, c6.y)};
  const ffv mz{make_float2(c5.x, c5.y), make_float2(c6.z, c6.w)};
  ffv d0 = v_diff(th[0], tl[0], pxh, pxl);
  ffv d1 = v_diff(th[1], tl[1], pyh, pyl);
  ffv d2 = v_diff(th[2], tl[2], pzh, pzl);
  ffv r2 = v_dot3(d0, d1, d2, d0, d1, d2);
  ffv ri = v_rsqrt(r2);
  ffv nd = v_dot3(mx, my, mz, d0, d1, d2);
  ffv ri2 = v_sq(ri);
  if (YUK) {
    ffv r = v_mul(r2, ri);
    ffv x = v_mul(kap, r);
    ffv e = v_expm(x, tab);
    ffv one_x = v_two_sum(vdup(1.0f), x.h);
    one_x = v_fast_two_sum(one_x.h, vadd(one_x.l, x.l));
    ffv t = v_add(ffv{sh, sl}, v_mul(v_mul(nd, one_x), ri2));
    return v_mul(t, v_mul(e, ri));
  }
  ffv t = v_add(ffv{sh, sl}, v_mul(nd, ri2));
  return v_mul(t, ri);
}

template <int NT, bool YUK>
__global__ void __launch_bounds__(NT) k_nbody_ff2(int nq, const float4* __restrict__ tgt,
                                                  const float4* __restrict__ src, float kh, float kl,
                                                  const float2* __restrict__ tab_hi, int per_split,
                                                  double* __restrict__ out) {
  __shared__ float4 shv[NT][7];   // duplicated (packed) copies
  __shared__ float4 shs[4][NT];   // scalar copies for the tiles that hold the thread's own targets
  __shared__ float2 tab[YUK ? FF_TABLE_HI : 1];
  if (YUK)
    for (int k = threadIdx.x; k < FF_TABLE_HI; k += NT) tab[k] = tab_hi[k];
  const int t0 = blockIdx.x * 2 * NT;
  const int i0 = t0 + threadIdx.x, i1 = t0 + NT + threadIdx.x;
  const int c0 = i0 < nq ? i0 : 0, c1 = i1 < nq ? i1 : 0;
  const float4 a0 = tgt[2 * c0], b0 = tgt[2 * c0 + 1];
  const float4 a1 = tgt[2 * c1], b1 = tgt[2 * c1 + 1];
  const float2 th[3] = {make_float2(a0.x, a1.x), make_float2(a0.y, a1.y), make_float2(a0.z, a1.z)};
  const float2 tl[3] = {make_float2(b0.x, b1.x), make_float2(b0.y, b1.y), make_float2(b0.z, b1.z)};
  const float ths0[3] = {a0.x, a0.y, a0.z}, tls0[3] = {b0.x, b0.y, b0.z};
  const float ths1[3] = {a1.x, a1.y, a1.z}, tls1[3] = {b1.x, b1.y, b1.z};
  const ffv kapv{vdup(kh), vdup(kl)};
  const ff kap{kh, kl};
  const int sb = blockIdx.y * per_split;
  const int se = min(nq, sb + per_split);
  double acc0 = 0.0, acc1 = 0.0;
  for (int s0 = sb; s0 < se; s0 += NT) {
    const int j = s0 + threadIdx.x;
    float4 c[4];
    if (j < se) {
      for (int k = 0; k < 4; ++k) c[k] = src[4 * j + k];
    } else {  // never read: the loops below stop at se
      c[0] = c[1] = c[2] = c[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int k = 0; k < 4; ++k) shs[k][threadIdx.x] = c[k];
    shv[threadIdx.x][0] = make_float4(c[0].x, c[0].x, c[0].y, c[0].y);
    shv[threadIdx.x][1] = make_float4(c[0].z, c[0].z, c[0].w, c[0].w);
    shv[threadIdx.x][2] = make_float4(c[1].x, c[1].x, c[1].y, c[1].y);
    shv[threadIdx.x][3] = make_float4(c[1].z, c[1].z, c[1].w, c[1].w);
    shv[threadIdx.x][4] = make_float4(c[2].x, c[2].x, c[2].y, c[2].y);
    shv[threadIdx.x][5] = make_float4(c[2].z, c[2].z, c[3].x, c[3].x);
    shv[threadIdx.x][6] = make_float4(c[3].y, c[3].y, c[3].z, c[3].z);
    __syncthreads();
    const int cnt = min(NT, se - s0);
    const bool diag = (s0 < t0 + 2 * NT) && (s0 + NT > t0);
    if (!diag) {
      ffv acc{vdup(0.f), vdup(0.f)};
      for (int jj = 0; jj < cnt; ++jj) acc = v_add(acc, v_pair<YUK>(shv[jj], th, tl, kapv, tab));
      acc0 += (double)acc.h.x + (double)acc.l.x;
      acc1 += (double)acc.h.y + (double)acc.l.y;
    } else {
      ff s0acc{0.f, 0.f}, s1acc{0.f, 0.f};
      for (int jj = 0; jj < cnt; ++jj) {
        if (s0 + jj != i0)
          s0acc = ff_add(s0acc, ff_pair<YUK>(shs[0][jj], shs[1][jj], shs[2][jj], shs[3][jj], ths0, tls0, kap, tab));
        if (s0 + jj != i1)
          s1acc = ff_add(s1acc, ff_pair<YUK>(shs[0][jj], shs[1][jj], shs[2][jj], shs[3][jj], ths1, tls1, kap, tab));
      }
      acc0 += (double)s0acc.h + (double)s0acc.l;
      acc1 += (double)s1acc.h + (double)s1acc.l;
    }
    __syncthreads();
  }
  if (i0 < nq) out[(int64_t)blockIdx.y * nq + i0] = acc0;
  if (i1 < nq) out[(int64_t)blockIdx.y * nq + i1] = acc1;
}

// Mutual float-float N-body: every unordered pair of points is evaluated once for both
// directions.  The pair (i, j) shares d = x_i - y_j, 1/r and, for the Yukawa kernel, exp(-kappa r);
// with f = (1 + kappa r) / r^2 and g = exp(-kappa r) / r it contributes
//   (s_j + (m_j . d) f) g  to target i   and   (s_i - (m_i . d) f) g  to target j,
// saving the shared part of the float-float work (about 30% of the operations).
//
// Points are cut into tiles of MT = 128 and the tiles into G groups; block (rg, cg), rg <= cg, takes
// every tile pair (I in rg, J in cg, I < J) and the diagonal tiles I = J (one direction, coincident
// point skipped).  Target-side sums stay in registers and go to PI[cg][i]; source-side sums are
// accumulated in shared memory per tile pair and added to PJ[rg][j], which only this block touches.
// Within a tile pair, step s of the 128 takes source 32 ((w + s / 32) mod 4) + (lane + s) mod 32 in
// warp w: the warps work on disjoint quarters of the source tile between barriers and the lanes of
// a warp on distinct sources, so the shared-memory sums have no races and a fixed order.  The
// final value of a point is the fixed-order sum of its 2 G partials (k_mutual_sum).
constexpr int MT = 128;

template <bool YUK>
__device__ __forceinline__ void ff_mutual(const float4& ah, const float4& al, const float4& amh, const float4& aml,
                                          const float4& bh, const float4& bl, const float4& bmh, const float4& bml,
                                          ff kap, const float2* __restrict__ tab, ff& to_a, ff& to_b) {
  // a = target (x, s, m), b = source (y, s, m); float4 (x, y, z, s) hi / lo, (mx, my, mz, -) hi / lo
  ff d0 = ff_diff(ah.x, al.x, bh.x, bl.x);
  ff d1 = ff_diff(ah.y, al.y, bh.y, bl.y);
  ff d2 = ff_diff(ah.z, al.z, bh.z, bl.z);
  ff r2 = ff_dot3(d0, d1, d2, d0, d1, d2);
  ff ri = ff_rsqrt(r2);
  ff ri2 = ff_sq(ri);
  ff f, g;
  if (YUK) {
    ff r = ff_mul(r2, ri);
    ff x = ff_mul(kap, r);
    ff e = ff_expm(x, tab);
    ff one_x = two_sum(1.0f, x.h);
    one_x = fast_two_sum(one_x.h, __fadd_rn(one_x.l, x.l));
    f = ff_mul(one_x, ri2);
    g = ff_mul(e, ri);
  } else {
    f = ri2;
    g = ri;
  }
  ff ndb = ff_dot3(ff{bmh.x, bml.x}, ff{bmh.y, bml.y}, ff{bmh.z, bml.z}, d0, d1, d2);
  ff nda = ff_dot3(ff{amh.x, aml.x}, ff{amh.y, aml.y}, ff{amh.z, aml.z}, d0, d1, d2);
  ff fb = ff_mul(ndb, f), fa = ff_mul(nda, f);
  to_a = ff_mul(ff_add(ff{bh.w, bl.w}, fb), g);
  to_b = ff_mul(ff_add(ff{ah.w, al.w}, ff{-fa.h, -fa.l}), g);
}

template <bool YUK>
__global__ void __launch_bounds__(MT) k_nbody_ffm(int nq, int G, const float4* __restrict__ src, float kh, float kl,
                                                  const float2* __restrict__ tab_hi, double* __restrict__ PI,
                                                  double* __restrict__ PJ) {
  __shared__ float4 sb[4][MT];              // source tile: (y, s) hi, (y, s) lo, m hi, m lo
  __shared__ float2 acc_j[MT];              // source-side float-float sums of the current tile pair
  __shared__ float2 tab[YUK ? FF_TABLE_HI : 1];
  if (YUK)
    for (int k = threadIdx.x; k < FF_TABLE_HI; k += MT) tab[k] = tab_hi[k];
  // block -> (rg, cg), rg <= cg
  int t = blockIdx.x, rg = 0;
  while (t >= G - rg) {
    t -= G - rg;
    ++rg;
  }
  const int cg = rg + t;
  const int nT = (nq + MT - 1) / MT;
  const int tpg = (nT + G - 1) / G;
  const int i0g = rg * tpg, i1g = min(nT, (rg + 1) * tpg);
  const int j0g = cg * tpg, j1g = min(nT, (cg + 1) * tpg);
  const ff kap{kh, kl};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int I = i0g; I < i1g; ++I) {
    const int i = I * MT + threadIdx.x;
    const bool iv = i < nq;
    // invalid targets sit far away with zero strength
    float4 ah = iv ? src[4 * i] : make_float4(2e15f, 0.f, 0.f, 0.f);
    float4 al = iv ? src[4 * i + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 amh = iv ? src[4 * i + 2] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 aml = iv ? src[4 * i + 3] : make_float4(0.f, 0.f, 0.f, 0.f);
    double acc64 = 0.0;
    for (int J = max(I, j0g); J < j1g; ++J) {
      const int jl = J * MT + threadIdx.x;
      __syncthreads();  // the previous tile's readers are done
      if (jl < nq) {
        for (int c = 0; c < 4; ++c) sb[c][threadIdx.x] = src[4 * jl + c];
      } else {
        sb[0][threadIdx.x] = make_float4(1e15f, 0.f, 0.f, 0.f);
        sb[1][threadIdx.x] = sb[2][threadIdx.x] = sb[3][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      acc_j[threadIdx.x] = make_float2(0.f, 0.f);
      __syncthreads();
      const int cnt = min(MT, nq - J * MT);
      ff acc{0.f, 0.f};
      if (J == I) {
        // diagonal tile: target side only, coincident point skipped
        const float th[3] = {ah.x, ah.y, ah.z}, tl[3] = {al.x, al.y, al.z};
        for (int jj = 0; jj < cnt; ++jj) {
          if (jj == (int)threadIdx.x) continue;
          acc = ff_add(acc, ff_pair<YUK>(sb[0][jj], sb[1][jj], sb[2][jj], sb[3][jj], th, tl, kap, tab));
        }
      } else {
        for (int ph = 0; ph < 4; ++ph) {
          const int base = 32 * ((warp + ph) & 3);
          for (int k = 0; k < 32; ++k) {
            const int jj = base + ((lane + k) & 31);
            ff ta, tb;
            ff_mutual<YUK>(ah, al, amh, aml, sb[0][jj], sb[1][jj], sb[2][jj], sb[3][jj], kap, tab, ta, tb);
            // running sums kept as (high, low) with the low parts and TwoSum errors added plainly
            // (at most 128 terms per tile pair, converted to float64 at its end)
            const ff sa = two_sum(acc.h, ta.h);
            acc = ff{sa.h, __fadd_rn(acc.l, __fadd_rn(sa.l, ta.l))};
            const float2 o = acc_j[jj];
            const ff sj = two_sum(o.x, tb.h);
            acc_j[jj] = make_float2(sj.h, __fadd_rn(o.y, __fadd_rn(sj.l, tb.l)));
            __syncwarp();
          }
          __syncthreads();
        }
        // source-side sums of this tile pair into PJ[rg][j]
        if (jl < nq) {
          const float2 o = acc_j[threadIdx.x];
          PJ[(int64_t)rg * nq + jl] += (double)o.x + (double)o.y;
        }
      }
      acc64 += (double)acc.h + (double)acc.l;
    }
    if (iv) PI[(int64_t)cg * nq + i] = acc64;
  }
}

// Packed mutual float-float N-body: k_nbody_ffm's pair organisation with two targets per thread
// on the float2 instructions.  Tiles hold MT2 = 256 points (targets i and i + 128 of a tile in one
// thread); a thread evaluates each source of the tile pair against both of its targets at once
// (the per-lane operation sequence of ff_mutual, so every pair value equals the scalar kernel's),
// adds the two lanes' source-side contributions and folds them into the tile's shared sums.  The
// 256 sources are visited in 8 chunks of 32: in phase p warp w takes chunk (w + p) mod 8 (the 4
// warps on distinct chunks between barriers) and lane l at step k source (l + k) mod 32 of it.
// Diagonal tiles take the scalar one-direction path with the coincident point skipped.
constexpr int MT2 = 2 * MT;

template <bool YUK>
__device__ __forceinline__ void v_mutual(const float2 (&ah)[3], const float2 (&al)[3], const ffv (&am)[3],
                                         const ffv& as, const float4& bh, const float4& bl, const float4& bmh,
                                         const float4& bml, ffv kap, const float2* __restrict__ tab, ffv& to_a,
                                         ffv& to_b) {
  ffv d0 = v_diff(ah[0], al[0], vdup(bh.x), vdup(bl.x));
  ffv d1 = v_diff(ah[1], al[1], vdup(bh.y), vdup(bl.y));
  ffv d2 = v_diff(ah[2], al[2], vdup(bh.z), vdup(bl.z));
  ffv r2 = v_dot3(d0, d1, d2, d0, d1, d2);
  ffv ri = v_rsqrt(r2);
  ffv ri2 = v_sq(ri);
  ffv f, g;
  if (YUK) {
    ffv r = v_mul(r2, ri);
    ffv x = v_mul(kap, r);
    ffv e = v_expm(x, tab);
    ffv one_x = v_two_sum(vdup(1.0f), x.h);
    one_x = v_fast_two_sum(one_x.h, vadd(one_x.l, x.l));
    f = v_mul(one_x, ri2);
    g = v_mul(e, ri);
  } else {
    f = ri2;
    g = ri;
  }
  ffv ndb = v_dot3(ffv{vdup(bmh.x), vdup(bml.x)}, ffv{vdup(bmh.y), vdup(bml.y)}, ffv{vdup(bmh.z), vdup(bml.z)}, d0,
                   d1, d2);
  ffv nda = v_dot3(am[0], am[1], am[2], d0, d1, d2);
  ffv fb = v_mul(ndb, f), fa = v_mul(nda, f);
  to_a = v_mul(v_add(ffv{vdup(bh.w), vdup(bl.w)}, fb), g);
  to_b = v_mul(v_add(as, ffv{vneg(fa.h), vneg(fa.l)}), g);
}

template <bool YUK>
__global__ void __launch_bounds__(MT) k_nbody_ffm2(int nq, int G, const float4* __restrict__ src, float kh,
                                                   float kl, const float2* __restrict__ tab_hi,
                                                   double* __restrict__ PI, double* __restrict__ PJ) {
  __shared__ float4 sb[4][MT2];             // source tile: (y, s) hi, (y, s) lo, m hi, m lo
  __shared__ float2 acc_j[MT2];             // source-side float-float sums of the current tile pair
  __shared__ float2 tab[YUK ? FF_TABLE_HI : 1];
  if (YUK)
    for (int k = threadIdx.x; k < FF_TABLE_HI; k += MT) tab[k] = tab_hi[k];
  int t = blockIdx.x, rg = 0;
  while (t >= G - rg) {
    t -= G - rg;
    ++rg;
  }
  const int cg = rg + t;
  const int nT = (nq + MT2 - 1) / MT2;
  const int tpg = (nT + G - 1) / G;
  const int i0g = rg * tpg, i1g = min(nT, (rg + 1) * tpg);
  const int j0g = cg * tpg, j1g = min(nT, (cg + 1) * tpg);
  const ff kap{kh, kl};
  const ffv kapv{vdup(kh), vdup(kl)};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int I = i0g; I < i1g; ++I) {
    const int i0 = I * MT2 + threadIdx.x, i1 = i0 + MT;
    const bool v0 = i0 < nq, v1 = i1 < nq;
    // invalid targets sit far away with zero strength
    const float4 a0h = v0 ? src[4 * i0] : make_float4(2e15f, 0.f, 0.f, 0.f);
    const float4 a0l = v0 ? src[4 * i0 + 1] : zero4;
    const float4 a0mh = v0 ? src[4 * i0 + 2] : zero4;
    const float4 a0ml = v0 ? src[4 * i0 + 3] : zero4;
    const float4 a1h = v1 ? src[4 * i1] : make_float4(2e15f, 0.f, 0.f, 0.f);
    const float4 a1l = v1 ? src[4 * i1 + 1] : zero4;
    const float4 a1mh = v1 ? src[4 * i1 + 2] : zero4;
    const float4 a1ml = v1 ? src[4 * i1 + 3] : zero4;
    const float2 ah[3] = {make_float2(a0h.x, a1h.x), make_float2(a0h.y, a1h.y), make_float2(a0h.z, a1h.z)};
    const float2 al[3] = {make_float2(a0l.x, a1l.x), make_float2(a0l.y, a1l.y), make_float2(a0l.z, a1l.z)};
    const ffv am[3] = {ffv{make_float2(a0mh.x, a1mh.x), make_float2(a0ml.x, a1ml.x)},
                       ffv{make_float2(a0mh.y, a1mh.y), make_float2(a0ml.y, a1ml.y)},
                       ffv{make_float2(a0mh.z, a1mh.z), make_float2(a0ml.z, a1ml.z)}};
    const ffv as{make_float2(a0h.w, a1h.w), make_float2(a0l.w, a1l.w)};
    double acc0 = 0.0, acc1 = 0.0;
    for (int J = max(I, j0g); J < j1g; ++J) {
      __syncthreads();  // the previous tile's readers are done
      for (int h = 0; h < 2; ++h) {
        const int slot = h * MT + threadIdx.x;
        const int jl = J * MT2 + slot;
        if (jl < nq) {
          for (int c = 0; c < 4; ++c) sb[c][slot] = src[4 * jl + c];
        } else {
          sb[0][slot] = make_float4(1e15f, 0.f, 0.f, 0.f);
          sb[1][slot] = sb[2][slot] = sb[3][slot] = zero4;
        }
        acc_j[slot] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (J == I) {
        // diagonal tile: target side only, coincident point skipped (scalar, per target)
        const int cnt = min(MT2, nq - J * MT2);
        for (int q = 0; q < 2; ++q) {
          const float4& xh = q == 0 ? a0h : a1h;
          const float4& xl = q == 0 ? a0l : a1l;
          const float th[3] = {xh.x, xh.y, xh.z}, tl[3] = {xl.x, xl.y, xl.z};
          const int self = q * MT + (int)threadIdx.x;
          ff acc{0.f, 0.f};
          for (int jj = 0; jj < cnt; ++jj) {
            if (jj == self) continue;
            acc = ff_add(acc, ff_pair<YUK>(sb[0][jj], sb[1][jj], sb[2][jj], sb[3][jj], th, tl, kap, tab));
          }
          (q == 0 ? acc0 : acc1) += (double)acc.h + (double)acc.l;
        }
      } else {
        ffv acc{vdup(0.f), vdup(0.f)};
        for (int ph = 0; ph < 8; ++ph) {
          const int base = 32 * ((warp + ph) & 7);
          for (int k = 0; k < 32; ++k) {
            const int jj = base + ((lane + k) & 31);
            ffv ta, tb;
            v_mutual<YUK>(ah, al, am, as, sb[0][jj], sb[1][jj], sb[2][jj], sb[3][jj], kapv, tab, ta, tb);
            // running sums kept as (high, low) with the low parts and TwoSum errors added plainly
            // (at most 256 terms per tile pair, converted to float64 at its end)
            const ffv sa = v_two_sum(acc.h, ta.h);
            acc = ffv{sa.h, vadd(acc.l, vadd(sa.l, ta.l))};
            const ff tbs = two_sum(tb.h.x, tb.h.y);
            const float tbl = __fadd_rn(tbs.l, __fadd_rn(tb.l.x, tb.l.y));
            const float2 o = acc_j[jj];
            const ff sj = two_sum(o.x, tbs.h);
            acc_j[jj] = make_float2(sj.h, __fadd_rn(o.y, __fadd_rn(sj.l, tbl)));
            __syncwarp();
          }
          __syncthreads();
        }
        // source-side sums of this tile pair into PJ[rg][j]
        for (int h = 0; h < 2; ++h) {
          const int slot = h * MT + threadIdx.x;
          const int jl = J * MT2 + slot;
          if (jl < nq) {
            const float2 o = acc_j[slot];
            PJ[(int64_t)rg * nq + jl] += (double)o.x + (double)o.y;
          }
        }
        acc0 += (double)acc.h.x + (double)acc.l.x;
        acc1 += (double)acc.h.y + (double)acc.l.y;
      }
    }
    if (v0) PI[(int64_t)cg * nq + i0] = acc0;
    if (v1) PI[(int64_t)cg * nq + i1] = acc1;
  }
}

// out[i] = sum over c of PI[c][i] + sum over r of PJ[r][i] (fixed order)
__global__ void k_mutual_sum(int nq, int G, const double* __restrict__ PI, const double* __restrict__ PJ,
                             double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  double v = 0.0;
  for (int c = 0; c < G; ++c) v += PI[(int64_t)c * nq + i];
  for (int r = 0; r < G; ++r) v += PJ[(int64_t)r * nq + i];
  out[i] = v;
}

// val[0][j] = sum over the source splits of val[split][j] (fixed order)
__global__ void k_split_sum(int nq, int nsplit, double* __restrict__ val) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nq || nsplit <= 1) return;
  double v = val[j];
  for (int sp = 1; sp < nsplit; ++sp) v += val[(int64_t)sp * nq + j];
  val[j] = v;
}

// y[i] (+)= scale * sum over incident (tau, a) of sum_q psi_a(x_q) w_q val[0][6 tau + q]; 4 lanes per vertex
__global__ void k_test_reduce(int nv, const int* __restrict__ ptr, const int* __restrict__ idx,
                              const double* __restrict__ val, int nsplit, int nq, const double* __restrict__ qw,
                              double scale, int accumulate, double* __restrict__ y) {
  const int lane = threadIdx.x & 3;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const bool valid = i < nv;  // all lanes reach the shuffles
  (void)nsplit;
  (void)nq;
  double acc = 0.0;
  const int b = valid ? ptr[i] : 0, e = valid ? ptr[i + 1] : 0;
  for (int k = b * QS + lane; k < e * QS; k += 4) {
    int ent = idx[k / QS], q = k % QS;
    int t = ent / 3, a = ent - 3 * t;
    int j = QS * t + q;
    acc += c_tri_b[q][a] * qw[j] * val[j];
  }
  acc += __shfl_down_sync(0xffffffffu, acc, 2, 4);
  acc += __shfl_down_sync(0xffffffffu, acc, 1, 4);
  if (lane == 0 && valid) {
    acc *= scale;
    y[i] = accumulate ? y[i] + acc : acc;
  }
}

// Coulomb sum at Gamma_m quadrature points: sum_k z_k / |x_j - x_k|.
__global__ void k_coulomb_qp(int nq, const double* __restrict__ qx, int ncharge, const double* __restrict__ cxyz,
                             const double* __restrict__ cz, double* __restrict__ out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nq) return;
  double x = qx[j], y = qx[nq + j], z = qx[2 * nq + j];
  double acc = 0.0;
  for (int k = 0; k < ncharge; ++k) {
    double dx = x - cxyz[k], dy = y - cxyz[ncharge + k], dz = z - cxyz[2 * ncharge + k];
    acc += cz[k] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  out[j] = acc;
}

// Reaction potential at the charges: (V_L lam)(x_k) - (K_L u)(x_k), 6-point rule (one block per charge).
// Reaction potentials of x_L and x_NL at the charges (Eq. Esolv's Gamma_m integral), both in one
// pass.  k_reaction_sources: per quadrature point j of Gamma_m its position, the normal of its
// triangle and, for both solutions, a_j = w_j lam_h(y_j) and c_j = w_j u_h(y_j) (9 values).
// k_reaction_pairs: block (charge k, chunk of points) sums a_j / r - c_j (n_j . d) / r^3 with
// d = x_k - y_j for both solutions (one float64 rsqrt per pair), one partial per block;
// k_reaction_sum adds a charge's chunk partials in chunk order and scales by 1/(4 pi).
constexpr int REAC_CHUNKS = 16;
constexpr int REAC_T = 256;

__global__ void k_reaction_sources(int nt, const int* __restrict__ tri, const int* __restrict__ vmap,
                                   const double* __restrict__ qx, const double* __restrict__ qw,
                                   const double* __restrict__ nrm, const double* __restrict__ lamL,
                                   const double* __restrict__ uL, const double* __restrict__ lamN,
                                   const double* __restrict__ uN, double* __restrict__ rec) {
  const int nq = QS * nt;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nq) return;
  const int t = j / QS, q = j - t * QS;
  double lL = 0.0, lU = 0.0, nL = 0.0, nU = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int v = tri[3 * t + a], sv = vmap[v];
    const double b = c_tri_b[q][a];
    lL += b * lamL[v];
    lU += b * uL[sv];
    nL += b * lamN[v];
    nU += b * uN[sv];
  }
  const double w = qw[j];
  rec[0 * (size_t)nq + j] = qx[j];
  rec[1 * (size_t)nq + j] = qx[nq + j];
  rec[2 * (size_t)nq + j] = qx[2 * nq + j];
  rec[3 * (size_t)nq + j] = nrm[t];
  rec[4 * (size_t)nq + j] = nrm[nt + t];
  rec[5 * (size_t)nq + j] = nrm[2 * nt + t];
  rec[6 * (size_t)nq + j] = w * lL;
  rec[7 * (size_t)nq + j] = w * lU;
  rec[8 * (size_t)nq + j] = w * nL;
  rec[9 * (size_t)nq + j] = w * nU;
}

__global__ void __launch_bounds__(REAC_T) k_reaction_pairs(int nq, const double* __restrict__ rec,
                                                           const double* __restrict__ cxyz, int ncharge,
                                                           double* __restrict__ part) {
  const int k = blockIdx.x, c = blockIdx.y;
  const double px = cxyz[k], py = cxyz[ncharge + k], pz = cxyz[2 * ncharge + k];
  const int per = (nq + REAC_CHUNKS - 1) / REAC_CHUNKS;
  const int j0 = c * per, j1 = min(nq, j0 + per);
  double accL = 0.0, accN = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += REAC_T) {
    const double dx = px - rec[j], dy = py - rec[(size_t)nq + j], dz = pz - rec[2 * (size_t)nq + j];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double ri = rsqrt(r2);
    const double ri3 = ri * ri * ri;
    const double nd = rec[3 * (size_t)nq + j] * dx + rec[4 * (size_t)nq + j] * dy + rec[5 * (size_t)nq + j] * dz;
    accL += rec[6 * (size_t)nq + j] * ri - rec[7 * (size_t)nq + j] * nd * ri3;
    accN += rec[8 * (size_t)nq + j] * ri - rec[9 * (size_t)nq + j] * nd * ri3;
  }
  __shared__ double sh[2][REAC_T / 32];
  accL = warp_sum(accL);
  accN = warp_sum(accN);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = accL;
    sh[1][threadIdx.x >> 5] = accN;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < REAC_T / 32; ++w) s += sh[threadIdx.x][w];
    part[((size_t)threadIdx.x * ncharge + k) * REAC_CHUNKS + c] = s;
  }
}

__global__ void k_reaction_sum(int n, const double* __restrict__ part, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < REAC_CHUNKS; ++c) s += part[(size_t)i * REAC_CHUNKS + c];
  out[i] = s * INV4PI;
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int init_quadrature() {
  static std::mutex mu;
  static bool done = false;
  std::lock_guard<std::mutex> lk(mu);
  if (done) return PBFB_OK;
  double x[NGL], w[NGL];
  gauss_legendre01(NGL, x, w);
  PB_CUDA(cudaMemcpyToSymbol(c_gl_x, x, sizeof(x)));
  PB_CUDA(cudaMemcpyToSymbol(c_gl_w, w, sizeof(w)));
  // 6-point rule on the 16 congruent sub-triangles of the 4-fold uniform refinement
  double sb[NSUB][3], sw[NSUB];
  int k = 0;
  const int m = 4;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m - i; ++j) {
      int cnt = (i + j < m - 1) ? 2 : 1;
      for (int up = 0; up < cnt; ++up) {
        int li[3][2];
        if (up == 0) {
          li[0][0] = i; li[0][1] = j; li[1][0] = i + 1; li[1][1] = j; li[2][0] = i; li[2][1] = j + 1;
        } else {
          li[0][0] = i + 1; li[0][1] = j; li[1][0] = i + 1; li[1][1] = j + 1; li[2][0] = i; li[2][1] = j + 1;
        }
        double cb[3][3];
        for (int c = 0; c < 3; ++c) {
          cb[c][0] = 1.0 - (li[c][0] + li[c][1]) / (double)m;
          cb[c][1] = li[c][0] / (double)m;
          cb[c][2] = li[c][1] / (double)m;
        }
        for (int q = 0; q < QS; ++q) {
          for (int d = 0; d < 3; ++d)
            sb[k][d] = h_tri_b[q][0] * cb[0][d] + h_tri_b[q][1] * cb[1][d] + h_tri_b[q][2] * cb[2][d];
          sw[k] = h_tri_w[q] / (m * m);
          ++k;
        }
      }
    }
  PB_CUDA(cudaMemcpyToSymbol(c_sub_b, sb, sizeof(sb)));
  PB_CUDA(cudaMemcpyToSymbol(c_sub_w, sw, sizeof(sw)));
  // float-float exp tables: exp(-k0 / 256), k0 < 16 (constant memory)
  float2 lo[16];
  for (int k = 0; k < 16; ++k) {
    double v = std::exp(-k / 256.0);
    float h = (float)v;
    lo[k] = make_float2(h, (float)(v - (double)h));
  }
  PB_CUDA(cudaMemcpyToSymbol(c_ff_exp_lo, lo, sizeof(lo)));
  done = true;
  return PBFB_OK;
}

// exp(-16 k1 / 256), k1 < FF_TABLE_HI, as float-float pairs (host-computed in float64)
int ff_exp_table(Mesh* m) {
  if (m->ff_tab.n) return PBFB_OK;
  std::vector<float2> t(FF_TABLE_HI);
  for (int k = 0; k < FF_TABLE_HI; ++k) {
    double v = std::exp(-16.0 * k / 256.0);
    float h = (float)v;
    t[k] = make_float2(h, (float)(v - (double)h));
  }
  PB_TRY(m->ff_tab.upload(t.data(), t.size(), m->stream));
  return PBFB_OK;
}

int test_reduce(Mesh* m, Surface* s, double* val, int nsplit, double* y, bool accumulate) {
  if (nsplit > 1) {
    k_split_sum<<<blocks_for(s->nq, 256), 256, 0, m->stream>>>(s->nq, nsplit, val);
    PB_LAUNCHED(m);
  }
  k_test_reduce<<<blocks_for((int64_t)s->nv * 4, 128), 128, 0, m->stream>>>(s->nv, s->inc_ptr.p, s->inc_idx.p, val,
                                                                            nsplit, s->nq, s->qw.p, 1.0,
                                                                            accumulate ? 1 : 0, y);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_surface_geometry(Mesh* m, Surface* s) {
  k_surface_geometry<<<blocks_for(s->nt, 128), 128, 0, m->stream>>>(
      m->xyz.p, m->nv, s->tri.p, s->vmap.p, s->nt, s->ctr[0], s->ctr[1], s->ctr[2], s->qx.p, s->qw.p, s->nrm.p,
      s->area.p, s->qpf.p);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int launch_pair_corrections(Mesh* m, Surface* s, double kappa) {
  if (s->npair == 0) return PBFB_OK;
  int threads = 128;
  int blocks = blocks_for((int64_t)s->npair * 32, threads);
  k_pair_corrections<<<blocks, threads, 0, m->stream>>>(
      s->npair, s->pair_t.p, s->pair_s.p, s->pair_cls.p, s->pair_perm.p, s->tri.p, s->vmap.p, m->xyz.p, m->nv,
      s->nrm.p, s->area.p, s->qx.p, s->qw.p, s->nt, kappa, s->pairV.p, s->pairK.p, s->pairVfull.p,
      m->red2.p);
  PB_LAUNCHED(m);
  // per-slot sums (fixed order): corrections, mass, V diagonal
  PB_TRY(launch_gather(m, s->cnnz, s->cg_ptr.p, s->cg_idx.p, s->pairV.p, nullptr, 1.0, s->corrV.p));
  PB_TRY(launch_gather(m, s->cnnz, s->cg_ptr.p, s->cg_idx.p, s->pairK.p, nullptr, 1.0, s->corrK.p));
  PB_TRY(launch_gather(m, s->cnnz, s->cg_ptr.p, s->cg_idx.p, m->red2.p, nullptr, 1.0, s->mass.p));
  PB_TRY(launch_gather(m, s->nv, s->dg_ptr.p, s->dg_idx.p, s->pairVfull.p, nullptr, 1.0, s->diagV.p));
  return PBFB_OK;
}

constexpr int F32_NT = 128;

// Launch shape of the float32 far field: tuning knobs if set, else 2 targets per thread with
// the packed kernel and 32 blocks per SM of source splits for large surfaces (GB300 sweep on
// the multi-charge sphere), one target per thread unpacked for small ones.
// With explicit targets per thread and blocks_per_sm 0, *bps = 0 asks the caller for a source
// split that fills whole waves of resident blocks.
void f32_shape(const Mesh* m, int nq, int* tpt, int* packed, int* bps) {
  const bool big = nq >= 16384;
  *tpt = m->tune_tpt > 0 ? m->tune_tpt : (big ? 2 : 1);
  *packed = m->tune_tpt > 0 ? m->tune_packed : (big ? 1 : 0);
  if (*tpt < 2 && *packed == 1) *packed = 0;
  *bps = m->tune_bps > 0 ? m->tune_bps : (m->tune_tpt > 0 ? 0 : (big ? 32 : 16));
}

// resident blocks per SM of the split float32 kernel variant
static int f32_blocks_per_sm(int tpt, int packed, bool yuk) {
  constexpr int NT = F32_NT;
  const void* f = nullptr;
  if (packed) {
    if (tpt == 2) f = yuk ? (const void*)k_nbody_f32x2<NT, 1, true> : (const void*)k_nbody_f32x2<NT, 1, false>;
    else if (tpt == 8) f = yuk ? (const void*)k_nbody_f32x2<NT, 4, true> : (const void*)k_nbody_f32x2<NT, 4, false>;
    else f = yuk ? (const void*)k_nbody_f32x2<NT, 2, true> : (const void*)k_nbody_f32x2<NT, 2, false>;
  } else {
    if (tpt == 1) f = yuk ? (const void*)k_nbody_f32<NT, 1, true> : (const void*)k_nbody_f32<NT, 1, false>;
    else if (tpt == 2) f = yuk ? (const void*)k_nbody_f32<NT, 2, true> : (const void*)k_nbody_f32<NT, 2, false>;
    else if (tpt == 8) f = yuk ? (const void*)k_nbody_f32<NT, 8, true> : (const void*)k_nbody_f32<NT, 8, false>;
    else f = yuk ? (const void*)k_nbody_f32<NT, 4, true> : (const void*)k_nbody_f32<NT, 4, false>;
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, NT, 0);
  return std::max(1, per);
}

void launch_nbody_f32(Mesh* m, Surface* s, double kappa, int tpt, int packed, int nsplit, int per,
                      const float4* spos, const float4* sdl, double* val) {
  constexpr int NT = F32_NT;
  const int nq = s->nq;
  const int ntb = blocks_for(nq, NT * tpt);
  dim3 grid(ntb, nsplit);
  const float kf = (float)kappa;
  const bool yuk = kappa != 0.0;
  const float4* q4 = s->qpf.p;
#define PB_NB(T)                                                                                    \
  if (yuk) k_nbody_f32<NT, T, true><<<grid, NT, 0, m->stream>>>(nq, q4, spos, sdl, kf, per, val);  \
  else k_nbody_f32<NT, T, false><<<grid, NT, 0, m->stream>>>(nq, q4, spos, sdl, kf, per, val);
#define PB_NB2(P)                                                                                   \
  if (yuk) k_nbody_f32x2<NT, P, true><<<grid, NT, 0, m->stream>>>(nq, q4, spos, sdl, kf, per, val); \
  else k_nbody_f32x2<NT, P, false><<<grid, NT, 0, m->stream>>>(nq, q4, spos, sdl, kf, per, val);
  if (packed) {
    switch (tpt) {
      case 2: PB_NB2(1) break;
      case 8: PB_NB2(4) break;
      default: PB_NB2(2) break;
    }
  } else {
    switch (tpt) {
      case 1: PB_NB(1) break;
      case 2: PB_NB(2) break;
      case 8: PB_NB(8) break;
      default: PB_NB(4) break;
    }
  }
#undef PB_NB
#undef PB_NB2
}

// y (+)= far-field part of the surface rows: for every test function psi_i,
//   sum_{x_q, y_p, q != p} psi_i(x_q) w_q [ g(x_q,y_p) s_p + dg/dn_y(x_q,y_p) m_p ]
// with s_p = cs w_p lam_h(y_p), m_p = cd w_p u_h(y_p) (kernel factors 1/(4 pi) included).
// lam indexed by local surface vertex; x (the shell part of the full vector, or a local
// surface vector when lam == x is a surface vector) indexed through vmap.
int launch_bem_far(Mesh* m, Surface* s, const double* x, const double* lam, double cs, double cd, double kappa,
                   int precision, double* y, bool accumulate) {
  const int nq = s->nq;
  const bool yuk = kappa != 0.0;
  const int u_local = (x != nullptr && x == lam) ? 1 : 0;
  const double* uvec = (cd != 0.0) ? x : nullptr;
  const double* lvec = (cs != 0.0) ? lam : nullptr;
  const bool f64 = precision == PBFB_FP64;
  if (precision == PBFB_FLOAT2) return launch_bem_far_ff(m, s, x, lam, cs, cd, kappa, y, accumulate);
  k_sources<<<blocks_for(nq, 256), 256, 0, m->stream>>>(s->nt, s->tri.p, s->vmap.p, lvec, uvec, u_local, s->qw.p,
                                                        s->nrm.p, s->qpf.p, s->qx.p, cs * INV4PI, cd * INV4PI,
                                                        f64 ? 1 : 0, s->spos.p, s->sdl.p, s->s64.p);
  PB_LAUNCHED(m);
  cudaEvent_t ev;
  KernelClassTimer& tm = f64 ? m->t_nbody64 : m->t_nbody;
  timer_begin(m, tm, &ev);
  int nsplit;
  double* vals = s->val.p;
  double tree_pairs = -1.0;
  if (f64) {
    constexpr int NT = 128;
    int ntb = blocks_for(nq, NT);
    nsplit = std::max(1, std::min(blocks_for(4 * 152, ntb), blocks_for(nq, 4 * NT)));
    int per = blocks_for(blocks_for(nq, nsplit), NT) * NT;
    nsplit = blocks_for(nq, per);
    dim3 grid(ntb, nsplit);
    if ((size_t)nsplit * nq > s->val.n) {
      set_error("far-field split buffer too small");
      return PBFB_ERR_STATE;
    }
    if (yuk)
      k_nbody_f64<NT, true><<<grid, NT, 0, m->stream>>>(nq, s->s64.p, kappa, per, s->val.p);
    else
      k_nbody_f64<NT, false><<<grid, NT, 0, m->stream>>>(nq, s->s64.p, kappa, per, s->val.p);
  } else if (use_tree(m, s)) {
    PB_TRY(launch_tree_far(m, s, kappa, s->spos.p, s->sdl.p, s->val.p, &tree_pairs));
    nsplit = 1;
  } else {
    int tpt, packed, bps;
    f32_shape(m, nq, &tpt, &packed, &bps);
    if (packed == 2) {
      // mutual pairs: G tile groups, G (G + 1) / 2 one-warp blocks (about bps per SM)
      const int nT = blocks_for(nq, FM_T);
      int G = (int)std::sqrt(2.0 * (bps > 0 ? bps : 32) * 152.0);
      G = std::max(1, std::min(G, nT));
      PB_TRY(ensure(s->mval, (size_t)(2 * G + 1) * nq));
      double* PI = s->mval.p;
      double* PJ = PI + (size_t)G * nq;
      double* out = PJ + (size_t)G * nq;
      PB_CUDA(cudaMemsetAsync(PI, 0, (size_t)2 * G * nq * sizeof(double), m->stream));
      const int nblk = G * (G + 1) / 2;
      if (yuk)
        k_nbody_f32m<true><<<nblk, 32, 0, m->stream>>>(nq, G, s->spos.p, s->sdl.p, (float)kappa, PI, PJ);
      else
        k_nbody_f32m<false><<<nblk, 32, 0, m->stream>>>(nq, G, s->spos.p, s->sdl.p, (float)kappa, PI, PJ);
      PB_LAUNCHED(m);
      k_mutual_sum<<<blocks_for(nq, 256), 256, 0, m->stream>>>(nq, G, PI, PJ, out);
      nsplit = 1;
      vals = out;
    } else {
      const int ntb = blocks_for(nq, F32_NT * tpt);
      if (bps == 0) {
        // whole waves: the largest split with at most 3 waves of resident blocks
        const int cap = f32_blocks_per_sm(tpt, packed, yuk) * 152;
        nsplit = std::max(1, std::min(3 * cap / ntb, blocks_for(nq, 4 * F32_NT)));
      } else {
        nsplit = std::max(1, std::min(blocks_for(bps * 152, ntb), blocks_for(nq, 4 * F32_NT)));
      }
      const int per = blocks_for(blocks_for(nq, nsplit), F32_NT) * F32_NT;
      nsplit = blocks_for(nq, per);
      if ((size_t)nsplit * nq > s->val.n) {
        set_error("far-field split buffer too small");
        return PBFB_ERR_STATE;
      }
      launch_nbody_f32(m, s, kappa, tpt, packed, nsplit, per, s->spos.p, s->sdl.p, s->val.p);
    }
  }
  PB_LAUNCHED(m);
  const double pairs = tree_pairs >= 0.0 ? tree_pairs : (double)nq * (double)nq;
  timer_end(m, tm, ev, pairs);
  if (!f64) m->nbody_flops += (yuk ? 24.0 : 18.0) * pairs;
  return test_reduce(m, s, vals, nsplit, y, accumulate);
}

int launch_bem_far_ff(Mesh* m, Surface* s, const double* x, const double* lam, double cs, double cd,
                      double kappa, double* y, bool accumulate) {
  const int nq = s->nq;
  const bool yuk = kappa != 0.0;
  const int u_local = (x != nullptr && x == lam) ? 1 : 0;
  PB_TRY(ff_exp_table(m));
  if (s->ffsrc.n < 4 * (size_t)nq) PB_TRY(s->ffsrc.alloc(4 * (size_t)nq));
  if (s->fftgt.n < 2 * (size_t)nq) PB_TRY(s->fftgt.alloc(2 * (size_t)nq));
  k_sources_ff<<<blocks_for(nq, 256), 256, 0, m->stream>>>(
      s->nt, s->tri.p, s->vmap.p, cs != 0.0 ? lam : nullptr, cd != 0.0 ? x : nullptr, u_local, s->qw.p, s->nrm.p,
      s->qx.p, s->ctr[0], s->ctr[1], s->ctr[2], cs * INV4PI, cd * INV4PI, s->ff_q, s->ffsrc.p, s->fftgt.p);
  PB_LAUNCHED(m);
  cudaEvent_t ev;
  timer_begin(m, m->t_nbodyff, &ev);
  constexpr int NT = 128;
  // kernel: 1 one target per thread, 2 two targets per thread (float2), 3 mutual pairs, 4 mutual
  // pairs with two targets per thread (float2);
  // built-in choice: packed mutual for large surfaces (5 % faster than 3 on GB300: the float32
  // pipe, not issue, bounds both), two targets per thread otherwise
  const int kind = m->tune_ff_kernel > 0 ? m->tune_ff_kernel : (nq >= 16384 ? 4 : 2);
  const int bps = m->tune_ff_bps > 0 ? m->tune_ff_bps : 8;  // GB300 sweep: 8 blocks per SM of source splits
  const float kh = (float)kappa, kl = (float)(kappa - (double)kh);
  if (kind == 3 || kind == 4) {
    // tile groups: G (G + 1) / 2 blocks, about bps blocks per SM (built-in 16: two waves, which
    // measured faster than one full wave or fewer, larger tiles); 2 G + 1 partial rows
    const int nT = blocks_for(nq, kind == 4 ? MT2 : MT);
    int G = (int)std::sqrt(2.0 * (m->tune_ff_bps > 0 ? m->tune_ff_bps : 16) * 152.0);
    G = std::max(1, std::min(G, nT));
    PB_TRY(ensure(s->mval, (size_t)(2 * G + 1) * nq));
    double* PI = s->mval.p;
    double* PJ = s->mval.p + (size_t)G * nq;
    double* out = s->mval.p + (size_t)2 * G * nq;
    PB_CUDA(cudaMemsetAsync(s->mval.p, 0, (size_t)2 * G * nq * sizeof(double), m->stream));
    const int nblk = G * (G + 1) / 2;
    if (kind == 4 && yuk)
      k_nbody_ffm2<true><<<nblk, MT, 0, m->stream>>>(nq, G, s->ffsrc.p, kh, kl, m->ff_tab.p, PI, PJ);
    else if (kind == 4)
      k_nbody_ffm2<false><<<nblk, MT, 0, m->stream>>>(nq, G, s->ffsrc.p, kh, kl, m->ff_tab.p, PI, PJ);
    else if (yuk)
      k_nbody_ffm<true><<<nblk, MT, 0, m->stream>>>(nq, G, s->ffsrc.p, kh, kl, m->ff_tab.p, PI, PJ);
    else
      k_nbody_ffm<false><<<nblk, MT, 0, m->stream>>>(nq, G, s->ffsrc.p, kh, kl, m->ff_tab.p, PI, PJ);
    PB_LAUNCHED(m);
    k_mutual_sum<<<blocks_for(nq, 256), 256, 0, m->stream>>>(nq, G, PI, PJ, out);
    PB_LAUNCHED(m);
    timer_end(m, m->t_nbodyff, ev, (double)nq * (double)nq);
    return test_reduce(m, s, out, 1, y, accumulate);
  }
  const bool pk = kind == 2;
  const int ntb = blocks_for(nq, pk ? 2 * NT : NT);
  // source splits from the packed grid in both variants, so that they sum in the same order
  const int ntb2 = blocks_for(nq, 2 * NT);
  int nsplit = std::max(1, std::min(blocks_for(bps * 152, ntb2), blocks_for(nq, 4 * NT)));
  const int per = blocks_for(blocks_for(nq, nsplit), NT) * NT;
  nsplit = blocks_for(nq, per);
  if ((size_t)nsplit * nq > s->val.n) {
    set_error("far-field split buffer too small");
    return PBFB_ERR_STATE;
  }
  dim3 grid(ntb, nsplit);
  if (pk && yuk)
    k_nbody_ff2<NT, true><<<grid, NT, 0, m->stream>>>(nq, s->fftgt.p, s->ffsrc.p, kh, kl, m->ff_tab.p, per, s->val.p);
  else if (pk)
    k_nbody_ff2<NT, false><<<grid, NT, 0, m->stream>>>(nq, s->fftgt.p, s->ffsrc.p, kh, kl, m->ff_tab.p, per, s->val.p);
  else if (yuk)
    k_nbody_ff<NT, true><<<grid, NT, 0, m->stream>>>(nq, s->fftgt.p, s->ffsrc.p, kh, kl, m->ff_tab.p, per, s->val.p);
  else
    k_nbody_ff<NT, false><<<grid, NT, 0, m->stream>>>(nq, s->fftgt.p, s->ffsrc.p, kh, kl, m->ff_tab.p, per, s->val.p);
  PB_LAUNCHED(m);
  timer_end(m, m->t_nbodyff, ev, (double)nq * (double)nq);
  return test_reduce(m, s, s->val.p, nsplit, y, accumulate);
}

int launch_coulomb(Mesh* m) {
  Surface* s = &m->sm;
  k_coulomb_qp<<<blocks_for(s->nq, 128), 128, 0, m->stream>>>(s->nq, s->qx.p, m->nq, m->qxyz.p, m->qz.p, s->val.p);
  PB_LAUNCHED(m);
  return test_reduce(m, s, s->val.p, 1, m->coul.p, false);
}

int launch_reaction_potentials(Mesh* m, const double* xL, const double* xNL, double* ur_dev) {
  Surface* s = &m->sm;
  if (m->nq == 0) return PBFB_OK;
  PB_TRY(ensure(m->reac_rec, 10 * (size_t)s->nq));
  PB_TRY(ensure(m->reac_part, 2 * (size_t)m->nq * REAC_CHUNKS));
  k_reaction_sources<<<blocks_for(s->nq, 256), 256, 0, m->stream>>>(s->nt, s->tri.p, s->vmap.p, s->qx.p, s->qw.p,
                                                                     s->nrm.p, xL + s->col0, xL, xNL + s->col0, xNL,
                                                                     m->reac_rec.p);
  PB_LAUNCHED(m);
  k_reaction_pairs<<<dim3(m->nq, REAC_CHUNKS), REAC_T, 0, m->stream>>>(s->nq, m->reac_rec.p, m->qxyz.p, m->nq,
                                                                       m->reac_part.p);
  PB_LAUNCHED(m);
  k_reaction_sum<<<blocks_for(2 * m->nq, 256), 256, 0, m->stream>>>(2 * m->nq, m->reac_part.p, ur_dev);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

}  // namespace pbfb

// ---------------------------------------------------------------- allocation-free far field
//
// pbfb_bem_apply_noalloc (include/pbfb.h) computes what pbfb_bem_apply computes with the
// float32 far field, but keeps all of its working memory in the fixed array below instead
// of buffers owned by the mesh: float32 source records (two float4 per quadrature point)
// followed by the float64 partial potentials of at most NOALLOC_SPLITS source splits.
// The array is a device global of the library: every device that loads libpbfb holds it
// until the process exits.  Calls share it, so calls that run at the same time on the GPU
// (other streams, other threads) overwrite each other's data.  Every call writes all of
// the scratch it reads, so nothing has to be cleared between calls.

namespace pbfb {
namespace {

constexpr int NOALLOC_MAX_QP = 65536;   // quadrature points (6 per triangle): 10922 triangles
constexpr int NOALLOC_SPLITS = 8;
constexpr size_t NOALLOC_BYTES =
    (size_t)NOALLOC_MAX_QP * 2 * sizeof(float4) + (size_t)NOALLOC_SPLITS * NOALLOC_MAX_QP * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device, looked up on the first call on that device.
// (In host code the symbol's name is only a host-side handle, not the device address.)  The
// entries are atomic: first calls from several host threads (server workers) may race to fill
// one; they all store the same address.
constexpr int NOALLOC_MAX_DEV = 64;
std::atomic<void*> g_noalloc_addr[NOALLOC_MAX_DEV];

int noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEV) {
    set_error("bem_apply_noalloc: device ordinal %d out of range", dev);
    return PBFB_ERR_INVALID;
  }
  void* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("bem_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return PBFB_ERR_CUDA;
    }
    g_noalloc_addr[dev].store(p, std::memory_order_release);
  }
  *out = (unsigned char*)p;
  return PBFB_OK;
}

}  // namespace

int bem_apply_noalloc(Mesh* m, int which, int op, const double* x, double* y) {
  Surface* s = which == PBFB_GAMMA_M ? &m->sm : &m->ss;
  const double kappa = which == PBFB_GAMMA_M ? 0.0 : m->kappa;
  const int nq = s->nq;
  if (nq > NOALLOC_MAX_QP) {
    set_error("bem_apply_noalloc: the surface has %d quadrature points; the fixed scratch holds at most %d "
              "(%d triangles)", nq, NOALLOC_MAX_QP, NOALLOC_MAX_QP / QS);
    return PBFB_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  PB_TRY(noalloc_scratch(m->dev, &base));
  float4* spos = (float4*)base;
  float4* sdl = spos + NOALLOC_MAX_QP;
  double* val = (double*)(sdl + NOALLOC_MAX_QP);
  const double cs = op == 0 ? 1.0 : 0.0, cd = op == 1 ? 1.0 : 0.0;
  k_sources<<<blocks_for(nq, 256), 256, 0, m->stream>>>(s->nt, s->tri.p, s->vmap.p, cs != 0.0 ? x : nullptr,
                                                        cd != 0.0 ? x : nullptr, 1, s->qw.p, s->nrm.p, s->qpf.p,
                                                        s->qx.p, cs * INV4PI, cd * INV4PI, 0, spos, sdl, nullptr);
  PB_LAUNCHED(m);
  // The split kernels and targets per thread of pbfb_bem_apply (launch_bem_far), with its split
  // rules (whole waves of resident blocks when blocks_per_sm is 0), capped at NOALLOC_SPLITS
  // source splits.  The mutual-pair variant (packed = 2) needs partial rows for every tile group,
  // more than the fixed array holds: it is replaced by the packed split kernel with the same
  // targets per thread, whose float32 sums run in another order.
  int tpt, packed, bps;
  f32_shape(m, nq, &tpt, &packed, &bps);
  if (packed == 2) {
    packed = tpt >= 2 ? 1 : 0;
    bps = 0;
  }
  const bool yuk = kappa != 0.0;
  const int ntb = blocks_for(nq, F32_NT * tpt);
  int nsplit;
  if (bps == 0) {
    const int cap = f32_blocks_per_sm(tpt, packed, yuk) * 152;
    nsplit = std::max(1, std::min(3 * cap / ntb, blocks_for(nq, 4 * F32_NT)));
  } else {
    nsplit = std::max(1, std::min(blocks_for(bps * 152, ntb), blocks_for(nq, 4 * F32_NT)));
  }
  nsplit = std::min(nsplit, NOALLOC_SPLITS);
  const int per = blocks_for(blocks_for(nq, nsplit), F32_NT) * F32_NT;
  nsplit = blocks_for(nq, per);
  launch_nbody_f32(m, s, kappa, tpt, packed, nsplit, per, spos, sdl, val);
  PB_LAUNCHED(m);
  PB_TRY(test_reduce(m, s, val, nsplit, y, false));
  PB_TRY(launch_csr_spmv(m, s->nv, s->c_ptr.p, s->c_col.p, op == 0 ? s->corrV.p : s->corrK.p, x, y, true));
  return PBFB_OK;
}

}  // namespace pbfb
