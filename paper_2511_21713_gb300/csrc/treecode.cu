// Hierarchical far field (treecode) for the float32 operator of GMRES.
//
// The paper switches its boundary operators from dense matrices to a fast multipole method for
// large surfaces (Sec. 3: above 90k vertices, order 3, leaves of fewer than 100 nodes).  Here the
// float32 quadrature-point sum of launch_bem_far,
//   phi(x_i) = sum_{j != i} [ s_j + m_j . (x_i - y_j) (1 + kappa r) / r^2 ] exp(-kappa r) / r,
// is split per target leaf B of a binary tree over the surface's quadrature points into
//   - near leaves, summed point by point (the leaf itself included, coincident points skipped),
//   - well-separated clusters C (r_B + r_C < theta |c_B - c_C|), each replaced by (p+1)^3 proxy
//     sources at the tensor Chebyshev points t_k (second kind) of its box, with charges
//     S_k = sum_{j in C} s_j L_k(y_j) and dipoles M_k = sum_{j in C} m_j L_k(y_j), where L_k is the
//     tensor barycentric Lagrange basis: the kernel's dependence on y is interpolated, so the
//     proxy sum is the same kernel evaluated at the proxies (barycentric Lagrange treecode of
//     Wang, Tlupova and Krasny, 2020).
// Both parts run through one kernel: a block takes one target leaf (up to 256 targets, two per
// thread, two sources per packed f32x2 operation) and a chunk of its source tiles (runs of at most 128
// consecutive source records: leaf points in tree order, or a cluster's proxies), and writes its
// partial sums; the chunks of a leaf are then added in a fixed order, so the result does not
// depend on scheduling.  The host plan (tree, acceptance, tiles, chunks) is built once per surface.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "f32x2.cuh"
#include "pbfb_internal.cuh"
#include "tree_plan.h"

namespace pbfb {

namespace {

constexpr int TREE_TILE = 128;               // source records per tile
constexpr int TREE_LEAF = 256;               // targets per leaf (at most)
constexpr int TREE_P = 6;                    // interpolation degree per dimension
constexpr int TREE_K = TREE_P + 1;           // Chebyshev points per dimension
constexpr int TREE_NPX = TREE_K * TREE_K * TREE_K;  // proxies per cluster
constexpr int TREE_UP_G = 8;                 // upward pass: point groups per (a, b) proxy column
constexpr int TREE_UP_NT = (TREE_K * TREE_K * TREE_UP_G + 31) / 32 * 32;  // threads of the upward pass
static_assert(TREE_UP_NT >= TREE_NPX && TREE_K <= 8, "upward pass shapes");
constexpr int TREE_TILES_PER_CHUNK = 8;      // source tiles per block
constexpr int TREE_EVAL_MINB = 8;            // evaluation blocks per SM the registers must allow (measured best)
constexpr double TREE_THETA = 0.6;           // acceptance: r_B + r_C < theta |c_B - c_C|

// tree order: spos_t[i] = spos[perm[i]] (sources and, for positions, the targets)
__global__ void k_tree_permute(int nq, const int* __restrict__ perm, const float4* __restrict__ spos,
                               const float4* __restrict__ sdl, float4* __restrict__ spos_t,
                               float4* __restrict__ sdl_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int j = perm[i];
  spos_t[i] = spos[j];
  sdl_t[i] = sdl[j];
}

// Upward pass, in two kernels.
// k_tree_up_leaf: a block per leaf (at most 256 points): proxy k = (a, b, c) at (tx_a, ty_b, tz_c) of
// the leaf's box receives sum_j L_a(x_j) L_b(y_j) L_c(z_j) (s_j, m_j) over the leaf's points, the
// 1-D values from the barycentric formula l_a(x) = (w_a / (x - t_a)) / sum_m (w_m / (x - t_m)),
// w_m = (-1)^m (halved at both ends), or the unit vector when x coincides with a node.  The basis
// values sit point-major in rows of 8 (lw[d][j][0..7]).  Thread t = 8 (a (p+1) + b) + g takes the
// column (a, b) -- all p+1 proxies c at once, from one product L_a L_b and two 16-byte reads of the
// row L_c -- over the points j = g mod 8; the 8 groups of a column are adjacent lanes and are added
// by a xor butterfly (every lane obtains the same sums).
// k_tree_m2c: a block per run of at most TREE_M2C_LEAVES consecutive leaves of one cluster: each
// leaf's proxies moved onto the cluster's Chebyshev grid, Q_C[k] += sum_k' L_k^C(s_k') Q_L[k'] --
// exact for the degree-p tensor basis L_k^C, so the cluster's proxies equal the sums over its points
// up to rounding -- as three passes of a (p+1) x (p+1) matrix, one dimension each, and added in leaf
// order.  The block that completes a cluster's last run (a per-cluster arrival counter) adds the
// cluster's runs in index order and writes its proxy
// source records, then re-arms the counter: the result does not depend on which block arrives last.
// Each point is touched once per solve-wide leaf instead of once per accepted ancestor.
__device__ __forceinline__ float cheb_node(const float* __restrict__ cbox, int c, int d, int k) {
  const float lo = cbox[6 * c + d], hi = cbox[6 * c + 3 + d];
  return 0.5f * (lo + hi) + 0.5f * (hi - lo) * cospif((float)k / (float)TREE_P);
}

// the p+1 barycentric Lagrange values at x of the nodes t[0..p] (unit vector on a node)
__device__ __forceinline__ void bary_row(float x, const float* t, float* l) {
  float a[TREE_K];
  float den = 0.f;
  int hit = -1;
#pragma unroll
  for (int k = 0; k < TREE_K; ++k) {
    const float dx = x - t[k];
    const float w = ((k & 1) ? -1.f : 1.f) * ((k == 0 || k == TREE_P) ? 0.5f : 1.f);
    if (dx == 0.f) hit = k;
    a[k] = dx == 0.f ? 0.f : w * rcp_approx(dx);
    den += a[k];
  }
  const float rden = rcp_approx(den);
#pragma unroll
  for (int k = 0; k < TREE_K; ++k) l[k] = hit >= 0 ? (k == hit ? 1.f : 0.f) : a[k] * rden;
}

__global__ void __launch_bounds__(TREE_UP_NT) k_tree_up_leaf(const int* __restrict__ leaf_beg,
                                                             const int* __restrict__ leaf_end,
                                                             const float* __restrict__ lbox,
                                                             const float4* __restrict__ pts_pos,
                                                             const float4* __restrict__ pts_dl,
                                                             float4* __restrict__ leaf_prox) {
  __shared__ float node[3][TREE_K];
  __shared__ __align__(16) float lw[3][TREE_LEAF][8];
  __shared__ float4 src[TREE_LEAF];
  const int L = blockIdx.x;
  const int b = leaf_beg[L], cnt = leaf_end[L] - b;
  const int t = threadIdx.x;
  if (t < 3 * TREE_K) node[t / TREE_K][t % TREE_K] = cheb_node(lbox, L, t / TREE_K, t % TREE_K);
  __syncthreads();
  for (int j = t; j < cnt; j += TREE_UP_NT) {
    const float4 p = pts_pos[b + j];
    const float4 q = pts_dl[b + j];
    src[j] = make_float4(p.w, q.x, q.y, q.z);
    const float xs[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float l[TREE_K];
      bary_row(xs[d], node[d], l);
#pragma unroll
      for (int k = 0; k < 8; ++k) lw[d][j][k] = k < TREE_K ? l[k] : 0.f;
    }
  }
  __syncthreads();
  const int col = t / TREE_UP_G, grp = t % TREE_UP_G;
  const bool colv = col < TREE_K * TREE_K;
  const int ka = colv ? col / TREE_K : 0, kb = colv ? col % TREE_K : 0;
  float acc[TREE_K][4];
#pragma unroll
  for (int k = 0; k < TREE_K; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
  if (colv) {
    for (int jj = grp; jj < cnt; jj += TREE_UP_G) {
      const float lab = lw[0][jj][ka] * lw[1][jj][kb];
      const float4 c0 = *reinterpret_cast<const float4*>(&lw[2][jj][0]);
      const float4 c1 = *reinterpret_cast<const float4*>(&lw[2][jj][4]);
      const float lc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      const float4 q = src[jj];
#pragma unroll
      for (int k = 0; k < TREE_K; ++k) {
        const float w = lab * lc[k];
        acc[k][0] = fmaf(w, q.x, acc[k][0]);
        acc[k][1] = fmaf(w, q.y, acc[k][1]);
        acc[k][2] = fmaf(w, q.z, acc[k][2]);
        acc[k][3] = fmaf(w, q.w, acc[k][3]);
      }
    }
  }
#pragma unroll
  for (int o = 1; o < TREE_UP_G; o <<= 1)
#pragma unroll
    for (int k = 0; k < TREE_K; ++k)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[k][v] += __shfl_xor_sync(0xffffffffu, acc[k][v], o);
  if (colv && grp == 0)
#pragma unroll
    for (int k = 0; k < TREE_K; ++k)
      leaf_prox[(size_t)L * TREE_NPX + col * TREE_K + k] = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
}

constexpr int TREE_M2C_NT = (TREE_NPX + 31) / 32 * 32;
constexpr int TREE_M2C_LEAVES = 4;  // leaves per block of k_tree_m2c

__global__ void __launch_bounds__(TREE_M2C_NT) k_tree_m2c(const int* __restrict__ pair_clus,
                                                          const int* __restrict__ pair_leaf,
                                                          const int* __restrict__ pair_nleaf,
                                                          const int* __restrict__ clus_pair,
                                                          const float* __restrict__ cbox,
                                                          const float* __restrict__ lbox,
                                                          const float4* __restrict__ leaf_prox,
                                                          float4* __restrict__ part, int* __restrict__ arrivals,
                                                          float4* __restrict__ prox_pos,
                                                          float4* __restrict__ prox_dl) {
  __shared__ float cn[3][TREE_K];
  __shared__ float mt[3][TREE_K][TREE_K];  // mt[d][a'][a] = l_a^C (the leaf's node a', dimension d)
  __shared__ float4 bufa[TREE_NPX], bufb[TREE_NPX];
  __shared__ int last;
  const int g = blockIdx.x;
  const int c = pair_clus[g], L0 = pair_leaf[g], nl = pair_nleaf[g];
  const int t = threadIdx.x;
  if (t < 3 * TREE_K) cn[t / TREE_K][t % TREE_K] = cheb_node(cbox, c, t / TREE_K, t % TREE_K);
  const int pa = t / (TREE_K * TREE_K), pb = (t / TREE_K) % TREE_K, pc = t % TREE_K;
  const bool tv = t < TREE_NPX;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int L = L0; L < L0 + nl; ++L) {
    __syncthreads();  // cn ready; the previous leaf's buffers consumed
    for (int i = t; i < TREE_NPX; i += TREE_M2C_NT) bufa[i] = leaf_prox[(size_t)L * TREE_NPX + i];
    if (t < 3 * TREE_K) {
      const int d = t / TREE_K, ap = t % TREE_K;
      float l[TREE_K];
      bary_row(cheb_node(lbox, L, d, ap), cn[d], l);
#pragma unroll
      for (int k = 0; k < TREE_K; ++k) mt[d][ap][k] = l[k];
    }
    __syncthreads();
    // x: bufb[a][b'][c'] = sum_a' mt[0][a'][a] bufa[a'][b'][c']
    if (tv) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int ap = 0; ap < TREE_K; ++ap) {
        const float w = mt[0][ap][pa];
        const float4 v = bufa[ap * TREE_K * TREE_K + pb * TREE_K + pc];
        s.x = fmaf(w, v.x, s.x);
        s.y = fmaf(w, v.y, s.y);
        s.z = fmaf(w, v.z, s.z);
        s.w = fmaf(w, v.w, s.w);
      }
      bufb[t] = s;
    }
    __syncthreads();
    // y: bufa[a][b][c'] = sum_b' mt[1][b'][b] bufb[a][b'][c']
    if (tv) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int bp = 0; bp < TREE_K; ++bp) {
        const float w = mt[1][bp][pb];
        const float4 v = bufb[pa * TREE_K * TREE_K + bp * TREE_K + pc];
        s.x = fmaf(w, v.x, s.x);
        s.y = fmaf(w, v.y, s.y);
        s.z = fmaf(w, v.z, s.z);
        s.w = fmaf(w, v.w, s.w);
      }
      bufa[t] = s;
    }
    __syncthreads();
    // z: this leaf's share of the cluster's proxies, added to the chunk's
    if (tv) {
#pragma unroll
      for (int cp = 0; cp < TREE_K; ++cp) {
        const float w = mt[2][cp][pc];
        const float4 v = bufa[pa * TREE_K * TREE_K + pb * TREE_K + cp];
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
        acc.z = fmaf(w, v.z, acc.z);
        acc.w = fmaf(w, v.w, acc.w);
      }
    }
  }
  if (tv) part[(size_t)g * TREE_NPX + t] = acc;
  // the last block of the cluster to arrive sums its pairs (release: fence before the count)
  __threadfence();
  __syncthreads();
  const int s0 = clus_pair[c], s1 = clus_pair[c + 1];
  if (t == 0) last = atomicAdd(&arrivals[c], 1) == s1 - s0 - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();  // acquire: the other pairs' partials are visible in L2
  if (tv) {
    // pair partials in batches of 8 independent loads, added in pair order
    double as = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    for (int h0 = s0; h0 < s1; h0 += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = h0 + u < s1 ? __ldcg(&part[(size_t)(h0 + u) * TREE_NPX + t]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (h0 + u < s1) {
          as += v[u].x;
          ax += v[u].y;
          ay += v[u].z;
          az += v[u].w;
        }
      }
    }
    const int o = c * TREE_NPX + t;
    prox_pos[o] = make_float4(cn[0][pa], cn[1][pb], cn[2][pc], (float)as);
    prox_dl[o] = make_float4((float)ax, (float)ay, (float)az, 0.f);
  }
  if (t == 0) arrivals[c] = 0;
}

// Evaluation: block = one chunk (a target leaf and a run of its source tiles of TREE_TILE records),
// TPT targets per thread (2: 128 threads; 4: 64 threads).  Tiles that overlap the leaf's own points
// take the scalar path with the coincident-point test; the others the packed one.  Padding entries
// (past a tile's count) sit far away with zero strength.
// Packed paths: a source tile sits in shared memory as one float array per record field, and a
// thread takes two consecutive sources at a time -- one 8-byte read per field is the f32x2 pack of
// both, every lane of the warp reading the same address -- against each of its targets held
// duplicated in both halves of a pack: per pair of sources and target one f32x2 operation does the
// work of two pairs.  (Reading one source duplicated into both halves, as the direct-sum kernels
// do, moves twice the shared-memory bytes per pair, and the shared-memory data path then bounds the
// kernel.)
// Coordinates of the packed paths: sources and targets relative to the centre c of the target
// leaf's box and, for the Yukawa kernel, multiplied by beta = kappa log2(e), so that
// e^{-kappa r} = 2^{-r'} with r' = beta r, d' = beta d and
//   [s + m.d (1/r + kappa)/r] e^{-kappa r}/r = beta [s + (beta m).d' (1/r' + ln 2)/r'] 2^{-r'}/r'
// (one multiplication per pair fewer; the factor beta is applied once per target at the end).
// Proxy tiles (sources at index >= nq) are well separated from the leaf: with r_B + r_C < theta D
// (D the distance of the box centres), |t'| < theta D, |y'| < (1 + theta) D and r > (1 - theta) D,
// so r'^2 = |t'|^2 + (|y'|^2 - 2 t'.y') and m'.d' = m'.t' - m'.y' lose at most a few units of
// float32 rounding to cancellation; they come from per-source fields (-2y', |y'|^2, m', -m'.y')
// in six float32 operations per pair fewer than the differences take.
enum { F_X, F_Y, F_Z, F_S, F_MX, F_MY, F_MZ, F_Q, F_P, F_N };  // shared-memory fields of a source tile

template <bool YUK, int TPT>
__global__ void __launch_bounds__(TREE_LEAF / TPT, TREE_EVAL_MINB) k_tree_eval(const float4* __restrict__ tgt_t,
                                                               const int* __restrict__ leaf_beg,
                                                               const int* __restrict__ leaf_end,
                                                               const float* __restrict__ lbox,
                                                               const int* __restrict__ chunk_leaf,
                                                               const int* __restrict__ chunk_tile,
                                                               const int2* __restrict__ tiles, int nq,
                                                               const float4* __restrict__ spos_t,
                                                               const float4* __restrict__ sdl_t, float kappa,
                                                               double* __restrict__ part) {
  constexpr int NT = TREE_LEAF / TPT;
  __shared__ __align__(16) float fld[F_N][TREE_TILE];
  __shared__ float4 shp[TREE_TILE], shd[TREE_TILE];
  const int c = blockIdx.x;
  const int L = chunk_leaf[c];
  const int lb = leaf_beg[L], le = leaf_end[L];
  const float cx = 0.5f * (lbox[6 * L] + lbox[6 * L + 3]), cy = 0.5f * (lbox[6 * L + 1] + lbox[6 * L + 4]),
              cz = 0.5f * (lbox[6 * L + 2] + lbox[6 * L + 5]);
  const float beta = YUK ? kappa * 1.4426950408889634f : 1.f;
  double acc64[TPT];
  f32x2 tx[TPT], ty[TPT], tz[TPT], tt2[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    acc64[k] = 0.0;
    const int i = lb + k * NT + threadIdx.x;
    const float4 p = tgt_t[i < le ? i : lb];
    const float x = (p.x - cx) * beta, y = (p.y - cy) * beta, z = (p.z - cz) * beta;
    tx[k] = pk2(x, x);
    ty[k] = pk2(y, y);
    tz[k] = pk2(z, z);
    const float t2 = fmaf(z, z, fmaf(y, y, x * x));
    tt2[k] = pk2(t2, t2);
  }
  const f32x2 ln2x2 = pk2(0.6931471805599453f, 0.6931471805599453f);
  for (int tl = chunk_tile[c]; tl < chunk_tile[c + 1]; ++tl) {
    const int2 tile = tiles[tl];
    const int s0 = tile.x, cnt = tile.y;
    const bool far = s0 >= nq;
    for (int i = threadIdx.x; i < TREE_TILE; i += NT) {
      float4 p, d;
      if (i < cnt) {
        p = spos_t[s0 + i];
        d = sdl_t[s0 + i];
      } else {
        p = make_float4(1e15f, 1e15f, 1e15f, 0.f);
        d = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const float yx = (p.x - cx) * beta, yy = (p.y - cy) * beta, yz = (p.z - cz) * beta;
      const float mx = d.x * beta, my = d.y * beta, mz = d.z * beta;
      if (far) {
        fld[F_X][i] = -2.f * yx;
        fld[F_Y][i] = -2.f * yy;
        fld[F_Z][i] = -2.f * yz;
        fld[F_Q][i] = fmaf(yz, yz, fmaf(yy, yy, yx * yx));
        fld[F_P][i] = -fmaf(mz, yz, fmaf(my, yy, mx * yx));
      } else {
        fld[F_X][i] = yx;
        fld[F_Y][i] = yy;
        fld[F_Z][i] = yz;
      }
      fld[F_S][i] = p.w;
      fld[F_MX][i] = mx;
      fld[F_MY][i] = my;
      fld[F_MZ][i] = mz;
      shp[i] = p;
      shd[i] = d;
    }
    __syncthreads();
    const bool diag = s0 < le && s0 + cnt > lb;
    if (!diag) {
      f32x2 acc[TPT];
#pragma unroll
      for (int k = 0; k < TPT; ++k) acc[k] = 0ull;
      if (far) {
#pragma unroll 2
        for (int jj = 0; jj < TREE_TILE; jj += 2) {
          const f32x2 X = *reinterpret_cast<const f32x2*>(&fld[F_X][jj]);
          const f32x2 Y = *reinterpret_cast<const f32x2*>(&fld[F_Y][jj]);
          const f32x2 Z = *reinterpret_cast<const f32x2*>(&fld[F_Z][jj]);
          const f32x2 Q = *reinterpret_cast<const f32x2*>(&fld[F_Q][jj]);
          const f32x2 MX = *reinterpret_cast<const f32x2*>(&fld[F_MX][jj]);
          const f32x2 MY = *reinterpret_cast<const f32x2*>(&fld[F_MY][jj]);
          const f32x2 MZ = *reinterpret_cast<const f32x2*>(&fld[F_MZ][jj]);
          const f32x2 P = *reinterpret_cast<const f32x2*>(&fld[F_P][jj]);
          const f32x2 S = *reinterpret_cast<const f32x2*>(&fld[F_S][jj]);
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const f32x2 r2 = add2(fma2(X, tx[k], fma2(Y, ty[k], fma2(Z, tz[k], Q))), tt2[k]);
            float ra, rb;
            upk2(r2, ra, rb);
            const f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
            const f32x2 nd = fma2(MX, tx[k], fma2(MY, ty[k], fma2(MZ, tz[k], P)));
            if (YUK) {
              float xa, xb;
              upk2(mul2(r2, ri), xa, xb);
              const f32x2 ex = pk2(ex2_approx(-xa), ex2_approx(-xb));
              const f32x2 tt = fma2(mul2(nd, ri), add2(ri, ln2x2), S);
              acc[k] = fma2(tt, mul2(ex, ri), acc[k]);
            } else {
              acc[k] = fma2(fma2(nd, mul2(ri, ri), S), ri, acc[k]);
            }
          }
        }
      } else {
#pragma unroll 2
        for (int jj = 0; jj < TREE_TILE; jj += 2) {
          const f32x2 X = *reinterpret_cast<const f32x2*>(&fld[F_X][jj]);
          const f32x2 Y = *reinterpret_cast<const f32x2*>(&fld[F_Y][jj]);
          const f32x2 Z = *reinterpret_cast<const f32x2*>(&fld[F_Z][jj]);
          const f32x2 MX = *reinterpret_cast<const f32x2*>(&fld[F_MX][jj]);
          const f32x2 MY = *reinterpret_cast<const f32x2*>(&fld[F_MY][jj]);
          const f32x2 MZ = *reinterpret_cast<const f32x2*>(&fld[F_MZ][jj]);
          const f32x2 S = *reinterpret_cast<const f32x2*>(&fld[F_S][jj]);
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const f32x2 dx = sub2(tx[k], X), dy = sub2(ty[k], Y), dz = sub2(tz[k], Z);
            const f32x2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            float ra, rb;
            upk2(r2, ra, rb);
            const f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
            const f32x2 nd = fma2(MZ, dz, fma2(MY, dy, mul2(MX, dx)));
            if (YUK) {
              float xa, xb;
              upk2(mul2(r2, ri), xa, xb);
              const f32x2 ex = pk2(ex2_approx(-xa), ex2_approx(-xb));
              const f32x2 tt = fma2(mul2(nd, ri), add2(ri, ln2x2), S);
              acc[k] = fma2(tt, mul2(ex, ri), acc[k]);
            } else {
              acc[k] = fma2(fma2(nd, mul2(ri, ri), S), ri, acc[k]);
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        float a, b;
        upk2(acc[k], a, b);
        acc64[k] += (double)a + (double)b;
      }
    } else {
      // the leaf's own points, in the original coordinates and units (scaled by 1 / beta here)
      const float nk = -kappa * 1.4426950408889634f;
      int ti[TPT];
      float txs[TPT], tys[TPT], tzs[TPT], accs[TPT];
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        ti[k] = lb + k * NT + threadIdx.x;
        const float4 p = tgt_t[ti[k] < le ? ti[k] : lb];
        txs[k] = p.x;
        tys[k] = p.y;
        tzs[k] = p.z;
        accs[k] = 0.f;
      }
      for (int jj = 0; jj < TREE_TILE; ++jj) {
        const float4 q = shp[jj];
        const float4 m = shd[jj];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
          if (s0 + jj == ti[k]) continue;
          const float dx = txs[k] - q.x, dy = tys[k] - q.y, dz = tzs[k] - q.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float ri = rsqrt_approx(r2);
          const float nd = fmaf(m.x, dx, fmaf(m.y, dy, m.z * dz));
          const float ri2 = ri * ri;
          if (YUK) {
            const float r = r2 * ri;
            const float ex = ex2_approx(nk * r);
            const float tt = fmaf(nd * fmaf(kappa, r, 1.f), ri2, q.w);
            accs[k] = fmaf(tt, ex * ri, accs[k]);
          } else {
            accs[k] = fmaf(fmaf(nd, ri2, q.w), ri, accs[k]);
          }
        }
      }
      const double ib = YUK ? 1.0 / (double)beta : 1.0;
#pragma unroll
      for (int k = 0; k < TPT; ++k) acc64[k] += (double)accs[k] * ib;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k)
    part[(size_t)c * TREE_LEAF + k * NT + threadIdx.x] = YUK ? acc64[k] * (double)beta : acc64[k];
}

// out[i] = in[perm[i]]
__global__ void k_tree_gather4(int nq, const int* __restrict__ perm, const float4* __restrict__ in,
                               float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nq) out[i] = in[perm[i]];
}

// val[perm[i]] = sum over the chunks of i's leaf, in chunk order
__global__ void k_tree_sum(int nq, const int* __restrict__ perm, const int* __restrict__ pos_leaf,
                           const int* __restrict__ leaf_beg, const int* __restrict__ leaf_chunk,
                           const double* __restrict__ part, double* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int L = pos_leaf[i];
  const int l = i - leaf_beg[L];
  // chunk partials in batches of 8 independent loads, added in chunk order
  double s = 0.0;
  const int c0 = leaf_chunk[L], c1 = leaf_chunk[L + 1];
  for (int cb = c0; cb < c1; cb += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = cb + u < c1 ? part[(size_t)(cb + u) * TREE_LEAF + l] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (cb + u < c1) s += v[u];
  }
  val[perm[i]] = s;
}

int blocks(int64_t n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

// Host plan of a surface's treecode (plan_tree_tiles: leaves of 256, splits at multiples of 256,
// clusters with more points than proxies), uploaded once per surface, on first use.
int build_surface_tree(Mesh* m, Surface* s) {
  SurfaceTree& T = s->tree;
  const int nq = s->nq;
  std::vector<double> qx(3 * (size_t)nq), xyz(3 * (size_t)nq);
  PB_CUDA(cudaMemcpyAsync(qx.data(), s->qx.p, qx.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PB_CUDA(cudaStreamSynchronize(m->stream));
  for (int j = 0; j < nq; ++j)
    for (int d = 0; d < 3; ++d) xyz[3 * (size_t)j + d] = qx[(size_t)d * nq + j];
  TreeTiles P;
  if (plan_tree_tiles(xyz.data(), nq, TREE_LEAF, TREE_THETA, TREE_NPX, TREE_TILE, TREE_TILES_PER_CHUNK, &P)) {
    set_error("treecode: tree plan failed");
    return PBFB_ERR_STATE;
  }
  // cluster boxes in the coordinates of the float32 records (relative to the surface centre)
  std::vector<float> cbox(P.clus_box.size());
  for (size_t k = 0; k < P.clus_box.size(); ++k) cbox[k] = (float)(P.clus_box[k] - s->ctr[k % 3]);
  std::vector<int2> tiles(P.tile_start.size());
  for (size_t t = 0; t < tiles.size(); ++t) tiles[t] = make_int2(P.tile_start[t], P.tile_count[t]);
  T.nq = nq;
  T.nleaf = P.nleaf;
  T.nclus = P.nclus;
  T.nchunk = (int)P.chunk_leaf.size();
  T.pairs = P.pairs;
  PB_TRY(T.perm.upload(P.perm.data(), nq, m->stream));
  PB_TRY(T.pos_leaf.upload(P.pos_leaf.data(), nq, m->stream));
  PB_TRY(T.leaf_beg.upload(P.leaf_beg.data(), P.nleaf, m->stream));
  PB_TRY(T.leaf_end.upload(P.leaf_end.data(), P.nleaf, m->stream));
  PB_TRY(T.leaf_chunk.upload(P.leaf_chunk.data(), P.leaf_chunk.size(), m->stream));
  PB_TRY(T.chunk_leaf.upload(P.chunk_leaf.data(), P.chunk_leaf.size(), m->stream));
  PB_TRY(T.chunk_tile.upload(P.chunk_tile.data(), P.chunk_tile.size(), m->stream));
  PB_TRY(T.tiles.upload(tiles.data(), tiles.size(), m->stream));
  // leaf boxes (the points' bounding boxes, a flat side widened to 1e-3 of the longest one, as the
  // clusters'): the upward pass's interpolation grids and the evaluation's coordinate origins
  {
    std::vector<float> lbox(6 * (size_t)P.nleaf);
    for (int L = 0; L < P.nleaf; ++L) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int q = P.leaf_beg[L]; q < P.leaf_end[L]; ++q)
        for (int d = 0; d < 3; ++d) {
          const double v = xyz[3 * (size_t)P.perm[q] + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
      double side = 0.0;
      for (int d = 0; d < 3; ++d) side = std::max(side, hi[d] - lo[d]);
      for (int d = 0; d < 3; ++d) {
        const double pad = std::max(0.0, 1e-3 * side - (hi[d] - lo[d])) * 0.5;
        lbox[6 * (size_t)L + d] = (float)(lo[d] - pad - s->ctr[d]);
        lbox[6 * (size_t)L + 3 + d] = (float)(hi[d] + pad - s->ctr[d]);
      }
    }
    PB_TRY(T.leaf_box.upload(lbox.data(), lbox.size(), m->stream));
  }
  if (P.nclus > 0) {
    // per cluster the leaves it is made of: clusters are tree nodes, unions of consecutive leaves
    // in tree order
    std::vector<int> pc, pl, pn, cp(1, 0);  // runs of leaves: cluster, first leaf, leaves
    for (int k = 0; k < P.nclus; ++k) {
      const int L0 = P.pos_leaf[P.clus_beg[k]], L1 = P.pos_leaf[P.clus_end[k] - 1];
      if (P.leaf_beg[L0] != P.clus_beg[k] || P.leaf_end[L1] != P.clus_end[k]) {
        set_error("treecode: a cluster is not a union of leaves");
        return PBFB_ERR_STATE;
      }
      for (int L = L0; L <= L1; L += TREE_M2C_LEAVES) {
        pc.push_back(k);
        pl.push_back(L);
        pn.push_back(std::min(TREE_M2C_LEAVES, L1 + 1 - L));
      }
      cp.push_back((int)pc.size());
    }
    T.npair = (int)pc.size();
    PB_TRY(T.clus_box.upload(cbox.data(), cbox.size(), m->stream));
    PB_TRY(T.pair_clus.upload(pc.data(), pc.size(), m->stream));
    PB_TRY(T.pair_leaf.upload(pl.data(), pl.size(), m->stream));
    PB_TRY(T.pair_nleaf.upload(pn.data(), pn.size(), m->stream));
    PB_TRY(T.clus_pair.upload(cp.data(), cp.size(), m->stream));
    PB_TRY(T.leaf_prox.alloc((size_t)P.nleaf * TREE_NPX));
    PB_TRY(T.up_part.alloc((size_t)T.npair * TREE_NPX));
    PB_TRY(T.up_arrivals.alloc(P.nclus));
    PB_CUDA(cudaMemsetAsync(T.up_arrivals.p, 0, P.nclus * sizeof(int), m->stream));
  }
  PB_TRY(T.spos.alloc((size_t)nq + (size_t)P.nclus * TREE_NPX));
  PB_TRY(T.sdl.alloc((size_t)nq + (size_t)P.nclus * TREE_NPX));
  PB_TRY(T.tgt.alloc(nq));
  PB_TRY(T.part.alloc((size_t)T.nchunk * TREE_LEAF));
  // target positions in tree order (the geometry does not change)
  k_tree_gather4<<<blocks(nq, 256), 256, 0, m->stream>>>(nq, T.perm.p, s->qpf.p, T.tgt.p);
  PB_LAUNCHED(m);
  PB_CUDA(cudaStreamSynchronize(m->stream));
  T.built = true;
  return PBFB_OK;
}

bool use_tree(const Mesh* m, const Surface* s) {
  if (m->tune_tree == 1) return false;
  if (m->tune_tree >= 2) return s->nq >= TREE_LEAF;
  return s->nq >= TREE_MIN_POINTS;
}

// float32 far field through the treecode: spos / sdl (original order, from k_sources) -> val
// (original order, one split).  Pair evaluations per call in *pairs.
int launch_tree_far(Mesh* m, Surface* s, double kappa, const float4* spos, const float4* sdl, double* val,
                    double* pairs) {
  SurfaceTree& T = s->tree;
  if (!T.built) PB_TRY(build_surface_tree(m, s));
  const int nq = s->nq;
  k_tree_permute<<<blocks(nq, 256), 256, 0, m->stream>>>(nq, T.perm.p, spos, sdl, T.spos.p, T.sdl.p);
  PB_LAUNCHED(m);
  if (T.nclus > 0) {
    k_tree_up_leaf<<<T.nleaf, TREE_UP_NT, 0, m->stream>>>(T.leaf_beg.p, T.leaf_end.p, T.leaf_box.p, T.spos.p,
                                                            T.sdl.p, T.leaf_prox.p);
    PB_LAUNCHED(m);
    k_tree_m2c<<<T.npair, TREE_M2C_NT, 0, m->stream>>>(T.pair_clus.p, T.pair_leaf.p, T.pair_nleaf.p, T.clus_pair.p,
                                                        T.clus_box.p, T.leaf_box.p, T.leaf_prox.p, T.up_part.p,
                                                        T.up_arrivals.p, T.spos.p + nq, T.sdl.p + nq);
    PB_LAUNCHED(m);
  }
  const float kf = (float)kappa;
  // four targets per thread with treecode = 3, else two.  The Yukawa form works in coordinates
  // scaled by kappa log2(e); below 1e-12 (no physical ionic strength) the kernel is the Laplace one
  // to far below float32 rounding (kappa r < 1e-9 here) and runs as such, keeping the scaled
  // squares clear of underflow.
  const bool four = m->tune_tree == 3;
  const bool yuk = kappa * 1.4426950408889634 >= 1e-12;
  const void* fn = yuk ? (four ? (const void*)k_tree_eval<true, 4> : (const void*)k_tree_eval<true, 2>)
                       : (four ? (const void*)k_tree_eval<false, 4> : (const void*)k_tree_eval<false, 2>);
  int nqa = nq;
  void* args[] = {&T.tgt.p,   &T.leaf_beg.p, &T.leaf_end.p, &T.leaf_box.p, &T.chunk_leaf.p, &T.chunk_tile.p,
                  &T.tiles.p, &nqa,          &T.spos.p,     &T.sdl.p,      (void*)&kf,      &T.part.p};
  PB_CUDA(cudaLaunchKernel(fn, dim3(T.nchunk), dim3(TREE_LEAF / (four ? 4 : 2)), args, 0, m->stream));
  PB_LAUNCHED(m);
  k_tree_sum<<<blocks(nq, 256), 256, 0, m->stream>>>(nq, T.perm.p, T.pos_leaf.p, T.leaf_beg.p, T.leaf_chunk.p,
                                                      T.part.p, val);
  PB_LAUNCHED(m);
  *pairs = T.pairs;
  return PBFB_OK;
}

}  // namespace pbfb
