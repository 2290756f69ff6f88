// Dense single-layer matrices of the two surfaces and their inverses, used on the surface
// rows of the block preconditioner of GMRES.  The paper solves every Newton increment
// (Sec. 2.4) with GMRES and does not state a preconditioner; this one is a design choice of
// this library.
//
// The diagonal blocks of the coupled operator on the unknowns lam_m and lam_s are -V_L
// (Gamma_m rows) and +V_Y (Gamma_s rows).  Scaling those rows by 1 / diag(V) leaves GMRES
// iterations growing with the condition number of V (like 1/h under refinement); applying
// V^-1 keeps them flat.  V is assembled densely in float32 from the same pieces as the
// matrix-free operator:
//   V = P^T G P + C
// with G the 6 x 6-point rule over all quadrature-point pairs (coincident points excluded),
// P the map from vertex values to weighted point values (w_q psi_i(x_q)), and C the sparse
// exact-minus-regular corrections of touching and near triangle pairs.  It is symmetrised
// and inverted in place by the sweep operator (Goodnight, "A tutorial on the SWEEP
// operator", The American Statistician 33, 1979) in pivot blocks of 64: sweeping every
// pivot of a symmetric positive definite matrix leaves -V^-1.
//
// Storage: row-major float32, leading dimension ld = n rounded up to 128; the padding rows
// and columns hold the identity, so every pivot block and update tile is full.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "pbfb_internal.cuh"
#include "quad_tables.cuh"

namespace pbfb {

namespace {

constexpr double INV4PI = 0.079577471545947667884;
constexpr int DW_T = 128;          // source vertices (threads) per block of the W kernel
constexpr int DW_A = 8;            // target points per block of the W kernel
constexpr int SW_B = 64;           // sweep pivot block
constexpr int SW_TILE = 128;       // update tile (and ld granularity)
constexpr size_t DENSE_W_BYTES = size_t(256) << 20;  // float32 work matrix W, per chunk

// W[a - a0][j] = sum over points b of the triangles around vertex j (b != a) of
//   w_b psi_j(y_b) g(x_a, y_b)
// for targets a in [a0, a0 + na).  Threads run over j; each block holds DW_A targets.
template <bool YUK>
__global__ void __launch_bounds__(DW_T) k_dense_w(int nv, int a0, int na, const float4* __restrict__ qpf,
                                                  const double* __restrict__ qw, const int* __restrict__ inc_ptr,
                                                  const int* __restrict__ inc_idx, float kappa,
                                                  float* __restrict__ W) {
  const int j = blockIdx.x * DW_T + threadIdx.x;
  const int ab = blockIdx.y * DW_A;
  float tx[DW_A], ty[DW_A], tz[DW_A], acc[DW_A];
#pragma unroll
  for (int u = 0; u < DW_A; ++u) {
    const float4 p = qpf[a0 + min(ab + u, na - 1)];
    tx[u] = p.x;
    ty[u] = p.y;
    tz[u] = p.z;
    acc[u] = 0.f;
  }
  if (j < nv) {
    for (int e = inc_ptr[j]; e < inc_ptr[j + 1]; ++e) {
      const int ent = inc_idx[e];
      const int t = ent / 3, k = ent - 3 * t;
      for (int q = 0; q < QS; ++q) {
        const int b = QS * t + q;
        const float4 p = qpf[b];
        const float wb = (float)(qw[b] * c_tri_b[q][k] * INV4PI);
#pragma unroll
        for (int u = 0; u < DW_A; ++u) {
          const float dx = tx[u] - p.x, dy = ty[u] - p.y, dz = tz[u] - p.z;
          // the coincident point gets r2 = 1e-30 (finite terms) and weight 0
          const float r2 = fmaxf(dx * dx + dy * dy + dz * dz, 1e-30f);
          const float ir = rsqrtf(r2);
          float g = (a0 + ab + u != b) ? ir : 0.f;
          if (YUK) g *= __expf(-kappa * r2 * ir);
          acc[u] += wb * g;
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < DW_A; ++u)
    if (j < nv && ab + u < na) W[(size_t)(ab + u) * nv + j] = acc[u];
}

// A[i][j] += sum over (tau, a) around vertex i with tau in [t0, t1) of
//   sum_q w_q psi_i(x_q) W[q-point of tau][j]
__global__ void k_dense_v(int nv, int ld, int t0, int t1, const float* __restrict__ W,
                          const double* __restrict__ qw, const int* __restrict__ inc_ptr,
                          const int* __restrict__ inc_idx, float* __restrict__ A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= nv) return;
  float acc = 0.f;
  bool any = false;
  for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; ++e) {
    const int ent = inc_idx[e];
    const int t = ent / 3, k = ent - 3 * t;
    if (t < t0 || t >= t1) continue;
    any = true;
    for (int q = 0; q < QS; ++q) {
      const int a = QS * t + q;
      acc += (float)(qw[a] * c_tri_b[q][k]) * W[(size_t)(a - QS * t0) * nv + j];
    }
  }
  if (any) A[(size_t)i * ld + j] += acc;
}

// zero, with the identity on the padding diagonal
__global__ void k_dense_init(int n, int ld, float* __restrict__ A) {
  const size_t tot = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e - (size_t)i * ld);
    A[e] = (i == j && i >= n) ? 1.f : 0.f;
  }
}

// sparse exact-minus-regular corrections, one thread per row
__global__ void k_dense_corr(int nv, int ld, const int* __restrict__ ptr, const int* __restrict__ col,
                             const double* __restrict__ corr, float* __restrict__ A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  for (int s = ptr[i]; s < ptr[i + 1]; ++s) A[(size_t)i * ld + col[s]] += (float)corr[s];
}

// A <- (A + A^T) / 2; the thread of (i, j > i) writes both entries
__global__ void k_dense_sym(int n, int ld, float* __restrict__ A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j <= i || j >= n) return;
  const float v = 0.5f * (A[(size_t)i * ld + j] + A[(size_t)j * ld + i]);
  A[(size_t)i * ld + j] = v;
  A[(size_t)j * ld + i] = v;
}

// Sweep of the SW_B x SW_B pivot block at (k0, k0), scalar pivots in order, in shared memory.
// Writes the swept block S (= -D, D the inverse of the block) and flags a pivot that is not
// positive and finite.
__global__ void __launch_bounds__(256) k_sweep_pivot(int ld, int k0, const float* __restrict__ A,
                                                     float* __restrict__ S, int* __restrict__ flag) {
  __shared__ float sS[SW_B][SW_B + 1];
  __shared__ float rowp[SW_B], colp[SW_B];
  const int tid = threadIdx.x;
  for (int e = tid; e < SW_B * SW_B; e += 256) {
    const int r = e / SW_B, c = e % SW_B;
    sS[r][c] = A[(size_t)(k0 + r) * ld + k0 + c];
  }
  __syncthreads();
  bool bad = false;
  for (int p = 0; p < SW_B; ++p) {
    if (tid < SW_B) {
      rowp[tid] = sS[p][tid];
      colp[tid] = sS[tid][p];
    }
    __syncthreads();
    const float d = rowp[p];
    bad = bad || !(d > 0.f) || !isfinite(d);
    const float inv = 1.f / d;
    for (int e = tid; e < SW_B * SW_B; e += 256) {
      const int r = e / SW_B, c = e % SW_B;
      sS[r][c] -= colp[r] * rowp[c] * inv;
    }
    __syncthreads();
    if (tid < SW_B) {
      sS[p][tid] = rowp[tid] * inv;
      sS[tid][p] = colp[tid] * inv;
    }
    __syncthreads();
    if (tid == 0) sS[p][p] = -inv;
    __syncthreads();
  }
  if (tid == 0 && bad) atomicExch(flag, 1);
  for (int e = tid; e < SW_B * SW_B; e += 256) {
    const int r = e / SW_B, c = e % SW_B;
    S[e] = sS[r][c];
  }
}

// Row panel of the pivot: P = A[K, :] (old values) and U = D P with D = -S; one column per thread.
// Only the tiles on and below the diagonal are kept current during the sweep (the matrix stays
// symmetric), so row K beyond its diagonal tile is read from column K: A[K][j] = A[j][K].
__global__ void __launch_bounds__(128) k_sweep_panel(int ld, int k0, const float* __restrict__ A,
                                                     const float* __restrict__ S, float* __restrict__ P,
                                                     float* __restrict__ U) {
  __shared__ float sD[SW_B][SW_B];
  for (int e = threadIdx.x; e < SW_B * SW_B; e += 128) sD[e / SW_B][e % SW_B] = -S[e];
  __syncthreads();
  const int j = blockIdx.x * 128 + threadIdx.x;  // ld is a multiple of 128
  const int kend = (k0 / SW_TILE + 1) * SW_TILE;  // end of the pivot's diagonal tile
  float pv[SW_B];
  if (j < kend) {
#pragma unroll
    for (int p = 0; p < SW_B; ++p) pv[p] = A[(size_t)(k0 + p) * ld + j];
  } else {
    const float4* col = reinterpret_cast<const float4*>(A + (size_t)j * ld + k0);
#pragma unroll
    for (int q = 0; q < SW_B / 4; ++q) {
      const float4 v = col[q];
      pv[4 * q] = v.x;
      pv[4 * q + 1] = v.y;
      pv[4 * q + 2] = v.z;
      pv[4 * q + 3] = v.w;
    }
  }
#pragma unroll
  for (int p = 0; p < SW_B; ++p) P[(size_t)p * ld + j] = pv[p];
  for (int p = 0; p < SW_B; ++p) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < SW_B; ++q) acc += sD[p][q] * pv[q];
    U[(size_t)p * ld + j] = acc;
  }
}

// Trailing update of one sweep step, 128 x 128 tiles on and below the diagonal (tile row >= tile
// column; the swept matrix is symmetric, the upper tiles are mirrored after the last step), 8 x 8
// per thread:
//   A[i][j] -= sum_p P[p][i] U[p][j]   (i, j outside K)
//   A[K][j] = U[:, j],  A[i][K] = U[:, i]^T,  A[K][K] = S
__global__ void __launch_bounds__(256) k_sweep_update(int ld, int k0, float* __restrict__ A,
                                                      const float* __restrict__ P, const float* __restrict__ U,
                                                      const float* __restrict__ S) {
  extern __shared__ float4 sm4[];
  float* Ps = reinterpret_cast<float*>(sm4);
  float* Us = Ps + SW_B * SW_TILE;
  const int tid = threadIdx.x;
  // blockIdx.x = I (I + 1) / 2 + J, J <= I
  int I = (int)((sqrtf(8.f * (float)blockIdx.x + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= (int)blockIdx.x) ++I;
  while (I * (I + 1) / 2 > (int)blockIdx.x) --I;
  const int J = (int)blockIdx.x - I * (I + 1) / 2;
  const int i0 = I * SW_TILE, j0 = J * SW_TILE;
  for (int e = tid; e < SW_B * SW_TILE / 4; e += 256) {
    const int p = e / (SW_TILE / 4), c4 = e % (SW_TILE / 4);
    reinterpret_cast<float4*>(Ps)[e] = *reinterpret_cast<const float4*>(P + (size_t)p * ld + i0 + 4 * c4);
    reinterpret_cast<float4*>(Us)[e] = *reinterpret_cast<const float4*>(U + (size_t)p * ld + j0 + 4 * c4);
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
#pragma unroll 4
  for (int p = 0; p < SW_B; ++p) {
    float a[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = Ps[p * SW_TILE + ty + 16 * r];
    const float4 b0 = *reinterpret_cast<const float4*>(Us + p * SW_TILE + 4 * tx);
    const float4 b1 = *reinterpret_cast<const float4*>(Us + p * SW_TILE + 64 + 4 * tx);
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] += a[r] * b[c];
  }
  const bool slow = (k0 >= i0 && k0 < i0 + SW_TILE) || (k0 >= j0 && k0 < j0 + SW_TILE);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + ty + 16 * r;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + 64 * h + 4 * tx;
      float4* dst = reinterpret_cast<float4*>(A + (size_t)i * ld + j);
      float4 o = *dst;
      float v[4] = {o.x - acc[r][4 * h], o.y - acc[r][4 * h + 1], o.z - acc[r][4 * h + 2], o.w - acc[r][4 * h + 3]};
      if (slow) {
        const unsigned di = (unsigned)(i - k0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const unsigned dj = (unsigned)(j + c - k0);
          if (di < SW_B && dj < SW_B)
            v[c] = S[di * SW_B + dj];
          else if (di < SW_B)
            v[c] = U[(size_t)di * ld + j + c];
          else if (dj < SW_B)
            v[c] = U[(size_t)dj * ld + i];
        }
      }
      *dst = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// Upper tiles from the lower ones after the sweep: A[j][i] = A[i][j] for tile row I > tile column J,
// through a 32 x 33 shared-memory transpose; block = one 32 x 32 sub-tile of a lower tile.
__global__ void k_sweep_mirror(int ld, float* __restrict__ A) {
  __shared__ float t[32][33];
  const int nt = ld / 32;
  const int b = blockIdx.x;  // lower sub-tiles (I > J) in row-major order
  int I = (int)((sqrtf(8.f * (float)b + 1.f) + 1.f) * 0.5f);
  while (I * (I - 1) / 2 > b) --I;
  while ((I + 1) * I / 2 <= b) ++I;
  const int J = b - I * (I - 1) / 2;
  if (I >= nt || J >= I) return;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) t[r][threadIdx.x] = A[(size_t)(32 * I + r) * ld + 32 * J + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) A[(size_t)(32 * J + r) * ld + 32 * I + threadIdx.x] = t[threadIdx.x][r];
}

// z[i] = scale * sum_j A[i][j] v[j], i < n: one warp per row, v staged in shared memory as float
__global__ void __launch_bounds__(256) k_dense_apply(int n, int ld, const float* __restrict__ A, double scale,
                                                     const double* __restrict__ v, double* __restrict__ z) {
  extern __shared__ float4 vs4[];
  float* vs = reinterpret_cast<float*>(vs4);
  for (int j = threadIdx.x; j < ld; j += 256) vs[j] = j < n ? (float)v[j] : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;  // the whole warp leaves together
  const float4* row = reinterpret_cast<const float4*>(A + (size_t)i * ld);
  float acc = 0.f;
  for (int c = lane; c < ld / 4; c += 32) {
    const float4 a = row[c];
    const float4 x = vs4[c];
    acc += a.x * x.x + a.y * x.y + a.z * x.z + a.w * x.w;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) z[i] = scale * (double)acc;
}

// out[i * ld_out + j] = scale * A[i * ld + j], i, j < n
__global__ void k_dense_copy(int n, int ld, const float* __restrict__ A, float scale, float* __restrict__ out,
                             int ld_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j < n) out[(size_t)i * ld_out + j] = scale * A[(size_t)i * ld + j];
}

int ensure_f(DBuf<float>& b, size_t n) {
  if (b.n >= n) return PBFB_OK;
  return b.alloc(n);
}

}  // namespace

int dense_ld(int n) { return (n + SW_TILE - 1) / SW_TILE * SW_TILE; }

size_t dense_bytes(int n) {
  const size_t ld = (size_t)dense_ld(n);
  return ld * ld * 4;
}

size_t dense_work_bytes(int n, int nt) {
  const size_t ld = (size_t)dense_ld(n);
  return std::min(DENSE_W_BYTES, (size_t)QS * nt * n * 4) + (2 * SW_B * ld + SW_B * SW_B + 64) * 4;
}

int build_dense_single_layer(Mesh* m, Surface* s, double kappa, bool invert) {
  const int n = s->nv, nt = s->nt;
  if (n < 1 || n > DENSE_V_MAX) {
    set_error("dense single layer: %d surface vertices (limit %d)", n, DENSE_V_MAX);
    return PBFB_ERR_INVALID;
  }
  if (s->kappa != kappa) {
    set_error("dense single layer: corrections were built for kappa %g, not %g", s->kappa, kappa);
    return PBFB_ERR_STATE;
  }
  const int ld = dense_ld(n);
  s->vinv_ok = false;
  PB_TRY(ensure_f(s->vinv, (size_t)ld * ld));
  s->vinv_ld = ld;
  // triangles per chunk of W (at most DENSE_W_BYTES of float32, released after the build)
  const int ct = (int)std::max<size_t>(1, std::min<size_t>(nt, DENSE_W_BYTES / ((size_t)QS * n * 4)));
  const size_t wlen = ((size_t)ct * QS * n + 63) / 64 * 64;  // keeps the panels 256-byte aligned
  PB_TRY(ensure_f(m->dwork, wlen + 2 * (size_t)SW_B * ld + SW_B * SW_B));
  if (m->dflag.n < 1) PB_TRY(m->dflag.alloc(1));
  float* W = m->dwork.p;
  float* P = W + wlen;
  float* U = P + (size_t)SW_B * ld;
  float* S = U + (size_t)SW_B * ld;
  float* A = s->vinv.p;
  cudaEvent_t ev;
  timer_begin(m, m->t_dense, &ev);
  k_dense_init<<<4 * 152, 256, 0, m->stream>>>(n, ld, A);
  PB_LAUNCHED(m);
  const dim3 gw((n + DW_T - 1) / DW_T, 1);
  if ((QS * ct + DW_A - 1) / DW_A > 65535) {
    set_error("dense single layer: work chunk too large");
    return PBFB_ERR_INVALID;
  }
  for (int t0 = 0; t0 < nt; t0 += ct) {
    const int t1 = std::min(nt, t0 + ct);
    const int na = QS * (t1 - t0);
    dim3 g(gw.x, (na + DW_A - 1) / DW_A);
    if (kappa != 0.0)
      k_dense_w<true><<<g, DW_T, 0, m->stream>>>(n, QS * t0, na, s->qpf.p, s->qw.p, s->inc_ptr.p, s->inc_idx.p,
                                                (float)kappa, W);
    else
      k_dense_w<false><<<g, DW_T, 0, m->stream>>>(n, QS * t0, na, s->qpf.p, s->qw.p, s->inc_ptr.p, s->inc_idx.p,
                                                 0.f, W);
    PB_LAUNCHED(m);
    k_dense_v<<<dim3(gw.x, n), DW_T, 0, m->stream>>>(n, ld, t0, t1, W, s->qw.p, s->inc_ptr.p, s->inc_idx.p, A);
    PB_LAUNCHED(m);
  }
  k_dense_corr<<<(n + 127) / 128, 128, 0, m->stream>>>(n, ld, s->c_ptr.p, s->c_col.p, s->corrV.p, A);
  PB_LAUNCHED(m);
  k_dense_sym<<<dim3(gw.x, n), DW_T, 0, m->stream>>>(n, ld, A);
  PB_LAUNCHED(m);
  if (invert) {
    PB_CUDA(cudaMemsetAsync(m->dflag.p, 0, sizeof(int), m->stream));
    const int smem = 2 * SW_B * SW_TILE * (int)sizeof(float);  // attribute set by init_dense_attributes
    const int ntile = ld / SW_TILE;
    const int gu = ntile * (ntile + 1) / 2;  // tiles on and below the diagonal
    for (int k0 = 0; k0 < ld; k0 += SW_B) {
      k_sweep_pivot<<<1, 256, 0, m->stream>>>(ld, k0, A, S, m->dflag.p);
      PB_LAUNCHED(m);
      k_sweep_panel<<<ld / 128, 128, 0, m->stream>>>(ld, k0, A, S, P, U);
      PB_LAUNCHED(m);
      k_sweep_update<<<gu, 256, smem, m->stream>>>(ld, k0, A, P, U, S);
      PB_LAUNCHED(m);
    }
    const int n32 = ld / 32;
    k_sweep_mirror<<<n32 * (n32 - 1) / 2, dim3(32, 8), 0, m->stream>>>(ld, A);
    PB_LAUNCHED(m);
    PB_CUDA(cudaMemcpyAsync(m->pinned, m->dflag.p, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  }
  timer_end(m, m->t_dense, ev, invert ? 2.0 * (double)ld * ld * ld : 0.0);
  PB_CUDA(cudaStreamSynchronize(m->stream));
  m->dwork.release();
  if (invert && reinterpret_cast<const int*>(m->pinned)[0] != 0) {
    set_error("dense single layer: a pivot of the float32 sweep was not positive");
    return PBFB_ERR_NONFINITE;
  }
  s->vinv_ok = invert;
  s->vinv_kappa = kappa;
  return PBFB_OK;
}

// Dynamic shared-memory limits of the dense kernels, set once per device by the first mesh
// creation, before any solve: the largest sweep tile pair, and the apply kernel's vector of
// dense_ld(DENSE_V_MAX) floats (every surface's fits).  Solves running on several host threads
// then never change a kernel's attributes while another thread launches or captures it, and a
// smaller matrix never lowers the limit a larger one needs.
int init_dense_attributes() {
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  PB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && ((done >> dev) & 1)) return PBFB_OK;
  PB_CUDA(cudaFuncSetAttribute(k_sweep_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               2 * SW_B * SW_TILE * (int)sizeof(float)));
  PB_CUDA(cudaFuncSetAttribute(k_dense_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               dense_ld(DENSE_V_MAX) * (int)sizeof(float)));
  if (dev < 64) done |= 1ull << dev;
  return PBFB_OK;
}

int launch_dense_apply(Mesh* m, Surface* s, double scale, const double* v, double* z) {
  if (!s->vinv_ok) {
    set_error("dense single-layer inverse not built");
    return PBFB_ERR_STATE;
  }
  const int smem = s->vinv_ld * (int)sizeof(float);  // within the limit of init_dense_attributes
  k_dense_apply<<<(s->nv + 7) / 8, 256, smem, m->stream>>>(s->nv, s->vinv_ld, s->vinv.p, scale, v, z);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

int dense_copy_out(Mesh* m, Surface* s, float scale, float* out, int ld_out) {
  k_dense_copy<<<dim3((s->nv + 127) / 128, s->nv), 128, 0, m->stream>>>(s->nv, s->vinv_ld, s->vinv.p, scale, out,
                                                                         ld_out);
  PB_LAUNCHED(m);
  return PBFB_OK;
}

}  // namespace pbfb
