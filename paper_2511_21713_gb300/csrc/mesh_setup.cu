// Mesh creation: validation, topology (host) and device data.
//
// The host builds integer structure only (CSR pattern of the coupled operator's sparse
// part, element-to-slot gather lists, triangle-pair classes); every floating-point
// quantity of the discretisation is computed on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pbfb_internal.cuh"
#include "quad_tables.cuh"

namespace pbfb {

namespace {

thread_local std::string g_err;

// counting sort of (key, value) pairs by key in [0, nkeys): returns ptr (nkeys+1) and values
void bucket(const std::vector<int>& keys, const std::vector<int>& vals, int nkeys, std::vector<int>& ptr,
            std::vector<int>& out) {
  ptr.assign(nkeys + 1, 0);
  for (int k : keys) ptr[k + 1]++;
  for (int i = 0; i < nkeys; ++i) ptr[i + 1] += ptr[i];
  out.resize(keys.size());
  std::vector<int> pos(ptr.begin(), ptr.end() - 1);
  for (size_t e = 0; e < keys.size(); ++e) out[pos[keys[e]]++] = vals[e];
}

struct HostSurface {
  std::vector<int> tri;    // local ids
  std::vector<int> verts;  // shell ids
  std::vector<double> P;   // nt*9 corner coordinates
};

// Triangle-pair classification (ordered pairs: test t, trial s): touching pairs (identical, common
// edge, common vertex) from the vertex incidence, near pairs (no common vertex, centroid distance
// below 2 max(h_t, h_s), h the longest edge) from a uniform grid over the centroids with cells of
// twice the median h.  A near pair is looked for from its triangle with the larger h (ties: the
// smaller index), within radius 2 h of that triangle, so every pair is found once whatever the
// spread of triangle sizes; host threads over the triangles.  Each row (test t) lists its trial
// triangles in ascending order.
void classify_pairs(const HostSurface& hs, std::vector<int>& pt, std::vector<int>& ps, std::vector<int>& cls,
                    std::vector<int>& perm) {
  const int nt = (int)hs.tri.size() / 3;
  const int nv = (int)hs.verts.size();
  std::vector<int> iptr(nv + 1, 0), inc(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) ++iptr[hs.tri[3 * t + a] + 1];
  for (int v = 0; v < nv; ++v) iptr[v + 1] += iptr[v];
  {
    std::vector<int> fill(iptr.begin(), iptr.end() - 1);
    for (int t = 0; t < nt; ++t)
      for (int a = 0; a < 3; ++a) inc[fill[hs.tri[3 * t + a]]++] = t;
  }
  std::vector<double> cen(3 * (size_t)nt), h(nt);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int t = 0; t < nt; ++t) {
    const double* P = &hs.P[9 * (size_t)t];
    double hh = 0.0;
    for (int d = 0; d < 3; ++d) cen[3 * (size_t)t + d] = (P[d] + P[3 + d] + P[6 + d]) / 3.0;
    for (int k = 0; k < 3; ++k) {
      const double* A = P + 3 * k;
      const double* B = P + 3 * ((k + 1) % 3);
      const double dx = B[0] - A[0], dy = B[1] - A[1], dz = B[2] - A[2];
      hh = std::max(hh, std::sqrt(dx * dx + dy * dy + dz * dz));
    }
    h[t] = hh;
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], cen[3 * (size_t)t + d]);
      hi[d] = std::max(hi[d], cen[3 * (size_t)t + d]);
    }
  }
  std::vector<double> hsort(h);
  std::nth_element(hsort.begin(), hsort.begin() + nt / 2, hsort.end());
  double cell = 2.0 * std::max(hsort[nt / 2], 1e-300);
  int dims[3];
  for (;;) {
    int64_t cells = 1;
    for (int d = 0; d < 3; ++d) {
      dims[d] = std::max(1, (int)std::floor((hi[d] - lo[d]) / cell) + 1);
      cells *= dims[d];
    }
    if (cells <= 8 * (int64_t)nt + 64) break;
    cell *= 2.0;
  }
  const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
  auto cidx = [&](double x, int d) { return std::min(dims[d] - 1, std::max(0, (int)std::floor((x - lo[d]) / cell))); };
  std::vector<int64_t> cptr(ncell + 1, 0);
  std::vector<int> ctri(nt), cof(nt);
  for (int t = 0; t < nt; ++t) {
    const double* c = &cen[3 * (size_t)t];
    cof[t] = (int)(((int64_t)cidx(c[0], 0) * dims[1] + cidx(c[1], 1)) * dims[2] + cidx(c[2], 2));
    ++cptr[cof[t] + 1];
  }
  for (int64_t k = 0; k < ncell; ++k) cptr[k + 1] += cptr[k];
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int t = 0; t < nt; ++t) ctri[fill[cof[t]]++] = t;
  }
  // near pairs, both orientations, from per-thread buffers merged in thread (= triangle) order
  const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::vector<int>> found(nth);
  auto search = [&](int k) {
    std::vector<int> stamp(nt, -1);
    std::vector<int>& out = found[k];
    const int t0 = (int)((int64_t)nt * k / nth), t1 = (int)((int64_t)nt * (k + 1) / nth);
    for (int t = t0; t < t1; ++t) {
      for (int a = 0; a < 3; ++a) {
        const int v = hs.tri[3 * t + a];
        for (int q = iptr[v]; q < iptr[v + 1]; ++q) stamp[inc[q]] = t;
      }
      const double* c = &cen[3 * (size_t)t];
      const double r = 2.0 * h[t];
      int a0[3], a1[3];
      for (int d = 0; d < 3; ++d) {
        a0[d] = cidx(c[d] - r, d);
        a1[d] = cidx(c[d] + r, d);
      }
      for (int x = a0[0]; x <= a1[0]; ++x)
        for (int y = a0[1]; y <= a1[1]; ++y)
          for (int z = a0[2]; z <= a1[2]; ++z) {
            const int64_t cc = ((int64_t)x * dims[1] + y) * dims[2] + z;
            for (int64_t q = cptr[cc]; q < cptr[cc + 1]; ++q) {
              const int u = ctri[q];
              if (stamp[u] == t) continue;  // itself and the touching triangles
              if (h[u] > h[t] || (h[u] == h[t] && u < t)) continue;  // found from u's side
              const double dx = c[0] - cen[3 * (size_t)u], dy = c[1] - cen[3 * (size_t)u + 1],
                           dz = c[2] - cen[3 * (size_t)u + 2];
              if (dx * dx + dy * dy + dz * dz < r * r) {
                out.push_back(t);
                out.push_back(u);
              }
            }
          }
    }
  };
  {
    std::vector<std::thread> th;
    for (int k = 1; k < nth; ++k) th.emplace_back(search, k);
    search(0);
    for (auto& x : th) x.join();
  }
  // rows: near partners of every triangle (both orientations), counting sort by row
  std::vector<int> nptr(nt + 1, 0);
  for (const auto& f : found)
    for (size_t q = 0; q < f.size(); q += 2) {
      ++nptr[f[q] + 1];
      ++nptr[f[q + 1] + 1];
    }
  for (int t = 0; t < nt; ++t) nptr[t + 1] += nptr[t];
  std::vector<int> near(nptr[nt]);
  {
    std::vector<int> fill(nptr.begin(), nptr.end() - 1);
    for (const auto& f : found)
      for (size_t q = 0; q < f.size(); q += 2) {
        near[fill[f[q]]++] = f[q + 1];
        near[fill[f[q + 1]]++] = f[q];
      }
  }
  std::vector<int> cnt(nt, 0), touched;
  std::vector<std::array<int, 2>> row;  // (s, class)
  for (int t = 0; t < nt; ++t) {
    touched.clear();
    row.clear();
    for (int a = 0; a < 3; ++a) {
      const int v = hs.tri[3 * t + a];
      for (int q = iptr[v]; q < iptr[v + 1]; ++q) {
        const int u = inc[q];
        if (cnt[u] == 0) touched.push_back(u);
        cnt[u]++;
      }
    }
    for (int u : touched) {
      const int c = cnt[u];
      row.push_back({u, c == 3 ? PAIR_IDENTICAL : (c == 2 ? PAIR_EDGE : PAIR_VERTEX)});
    }
    for (int q = nptr[t]; q < nptr[t + 1]; ++q) row.push_back({near[q], PAIR_NEAR});
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      int u = e[0], c = e[1];
      int p[6] = {0, 1, 2, 0, 1, 2};
      const int* T = &hs.tri[3 * t];
      const int* S = &hs.tri[3 * u];
      if (c == PAIR_EDGE) {
        // shared vertices in the test triangle's order go to reference vertices 0 and 1
        int sh[2], ns = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (T[a] == S[b]) sh[ns++] = a;
        int sb[2];
        for (int k = 0; k < 2; ++k)
          for (int b = 0; b < 3; ++b)
            if (S[b] == T[sh[k]]) sb[k] = b;
        p[0] = sh[0]; p[1] = sh[1]; p[2] = 3 - sh[0] - sh[1];
        p[3] = sb[0]; p[4] = sb[1]; p[5] = 3 - sb[0] - sb[1];
      } else if (c == PAIR_VERTEX) {
        int ia = 0, ib = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (T[a] == S[b]) { ia = a; ib = b; }
        for (int k = 0; k < 3; ++k) {
          p[k] = (ia + k) % 3;
          p[3 + k] = (ib + k) % 3;
        }
      }
      pt.push_back(t);
      ps.push_back(u);
      cls.push_back(c);
      for (int k = 0; k < 6; ++k) perm.push_back(p[k]);
    }
    for (int u : touched) cnt[u] = 0;
  }
}

int build_surface(Mesh* m, Surface* s, const std::vector<int>& gtri, const std::vector<double>& xyz_h) {
  const int nt = (int)gtri.size() / 3;
  std::vector<int> verts(gtri.begin(), gtri.end());
  std::sort(verts.begin(), verts.end());
  verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
  std::unordered_map<int, int> loc;
  for (int i = 0; i < (int)verts.size(); ++i) loc[verts[i]] = i;
  HostSurface hs;
  hs.verts = verts;
  hs.tri.resize(gtri.size());
  hs.P.resize(9 * (size_t)nt);
  double c[3] = {0, 0, 0};
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      int g = gtri[3 * t + a];
      hs.tri[3 * t + a] = loc[g];
      for (int d = 0; d < 3; ++d) hs.P[9 * t + 3 * a + d] = xyz_h[3 * (size_t)g + d];
    }
  for (int v : verts)
    for (int d = 0; d < 3; ++d) c[d] += xyz_h[3 * (size_t)v + d];
  for (int d = 0; d < 3; ++d) s->ctr[d] = c[d] / verts.size();
  {
    // float-float coordinates: high parts on the grid 2^-k with every difference of two high
    // parts below 2^24 steps, hence exact in float32 (quadrature points lie within the
    // triangles, so within the largest vertex distance from the centre)
    double rmax = 0.0;
    for (int v : verts) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double x = xyz_h[3 * (size_t)v + d] - s->ctr[d];
        r2 += x * x;
      }
      rmax = std::max(rmax, std::sqrt(r2));
    }
    const int k = (int)std::floor(24.0 - std::log2(2.0 * rmax * 1.01 + 1e-300)) - 1;
    s->ff_q = std::ldexp(1.0, -k);
  }
  s->nt = nt;
  s->nv = (int)verts.size();
  s->nq = QS * nt;
  s->tri_h = hs.tri;
  s->vmap_h = verts;
  PB_TRY(s->tri.upload(hs.tri.data(), hs.tri.size(), m->stream));
  PB_TRY(s->vmap.upload(verts.data(), verts.size(), m->stream));
  // test-reduction incidence: per vertex (t*3 + a)
  {
    std::vector<int> keys, vals;
    for (int t = 0; t < nt; ++t)
      for (int a = 0; a < 3; ++a) {
        keys.push_back(hs.tri[3 * t + a]);
        vals.push_back(3 * t + a);
      }
    std::vector<int> ptr, out;
    bucket(keys, vals, s->nv, ptr, out);
    PB_TRY(s->inc_ptr.upload(ptr.data(), ptr.size(), m->stream));
    PB_TRY(s->inc_idx.upload(out.data(), out.size(), m->stream));
  }
  // special pairs and the correction pattern
  std::vector<int> pt, ps, cls, perm;
  classify_pairs(hs, pt, ps, cls, perm);
  s->npair = (int)pt.size();
  PB_TRY(s->pair_t.upload(pt.data(), pt.size(), m->stream));
  PB_TRY(s->pair_s.upload(ps.data(), ps.size(), m->stream));
  PB_TRY(s->pair_cls.upload(cls.data(), cls.size(), m->stream));
  PB_TRY(s->pair_perm.upload(perm.data(), perm.size(), m->stream));
  {
    // entry e = 9 p + 3 a + b of pair p couples test vertex tri[pt[p]][a] and trial vertex
    // tri[ps[p]][b]; rows by counting sort, then columns sorted within each row
    const size_t ne = 9 * (size_t)s->npair;
    std::vector<int> rows(ne), vals(ne), slot_of(ne), dk, dv;
    for (size_t e = 0; e < ne; ++e) {
      const int p = (int)(e / 9), a = (int)(e / 3) % 3, b = (int)(e % 3);
      rows[e] = hs.tri[3 * pt[p] + a];
      vals[e] = (int)e;
      if (rows[e] == hs.tri[3 * ps[p] + b]) {
        dk.push_back(rows[e]);
        dv.push_back((int)e);
      }
    }
    std::vector<int> colv(ne);
    for (size_t e = 0; e < ne; ++e) colv[e] = hs.tri[3 * ps[e / 9] + e % 3];
    std::vector<int> rptr, rent;
    bucket(rows, vals, s->nv, rptr, rent);
    s->c_ptr_h.assign(s->nv + 1, 0);
    s->c_col_h.clear();
    // per row: the distinct columns in first-seen order (a marker per column), sorted, then every
    // entry's slot is its column's rank in the row
    std::vector<int> mark(s->nv, -1), distinct;
    for (int i = 0; i < s->nv; ++i) {
      distinct.clear();
      for (int q = rptr[i]; q < rptr[i + 1]; ++q) {
        const int c = colv[rent[q]];
        if (mark[c] < 0) {
          mark[c] = 0;
          distinct.push_back(c);
        }
      }
      std::sort(distinct.begin(), distinct.end());
      const int base = (int)s->c_col_h.size();
      for (size_t r = 0; r < distinct.size(); ++r) {
        mark[distinct[r]] = base + (int)r;
        s->c_col_h.push_back(distinct[r]);
      }
      for (int q = rptr[i]; q < rptr[i + 1]; ++q) slot_of[rent[q]] = mark[colv[rent[q]]];
      for (int c : distinct) mark[c] = -1;
      s->c_ptr_h[i + 1] = (int)s->c_col_h.size();
    }
    s->cnnz = (int)s->c_col_h.size();
    std::vector<int> ptr, out;
    bucket(slot_of, vals, s->cnnz, ptr, out);
    PB_TRY(s->cg_ptr.upload(ptr.data(), ptr.size(), m->stream));
    PB_TRY(s->cg_idx.upload(out.data(), out.size(), m->stream));
    bucket(dk, dv, s->nv, ptr, out);
    PB_TRY(s->dg_ptr.upload(ptr.data(), ptr.size(), m->stream));
    PB_TRY(s->dg_idx.upload(out.data(), out.size(), m->stream));
    PB_TRY(s->c_ptr.upload(s->c_ptr_h.data(), s->c_ptr_h.size(), m->stream));
    PB_TRY(s->c_col.upload(s->c_col_h.data(), s->c_col_h.size(), m->stream));
  }
  PB_TRY(s->qx.alloc(3 * (size_t)s->nq));
  PB_TRY(s->qw.alloc(s->nq));
  PB_TRY(s->nrm.alloc(3 * (size_t)nt));
  PB_TRY(s->area.alloc(nt));
  PB_TRY(s->qpf.alloc(s->nq));
  PB_TRY(s->pairV.alloc(9 * (size_t)s->npair));
  PB_TRY(s->pairK.alloc(9 * (size_t)s->npair));
  PB_TRY(s->pairVfull.alloc(9 * (size_t)s->npair));
  PB_TRY(s->corrV.alloc(s->cnnz));
  PB_TRY(s->corrK.alloc(s->cnnz));
  PB_TRY(s->mass.alloc(s->cnnz));
  PB_TRY(s->diagV.alloc(s->nv));
  PB_TRY(s->spos.alloc(s->nq));
  PB_TRY(s->sdl.alloc(s->nq));
  PB_TRY(s->s64.alloc(7 * (size_t)s->nq));
  // far-field partial-sum buffer: enough source splits for every launch shape of launch_bem_far
  PB_TRY(s->val.alloc(far_splits_max(s->nq) * (size_t)s->nq));
  return PBFB_OK;
}

int64_t key2(int r, int c) { return ((int64_t)r << 32) | (uint32_t)c; }

}  // namespace

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

const char* last_error() { return g_err.c_str(); }

// Validation of the shell mesh and its two boundary surfaces (host).
// With region (per tet 0 = Omega_m, 1 = Omega_i), Gamma_m must be the interface between the two
// regions (interior faces, normal into Omega_i) and Gamma_s the whole boundary.
static int validate(const double* xyz, int nv, const int* tets, int64_t nt, const int* gm, int ngm, const int* gs,
                    int ngs, const int* region) {
  if (!xyz || !tets || !gm || !gs || nv < 4 || nt < 1 || ngm < 4 || ngs < 4) {
    set_error("mesh_create: empty or missing arrays");
    return PBFB_ERR_INVALID;
  }
  if (nt > (int64_t(1) << 29)) {
    set_error("mesh_create: more than 2^29 tetrahedra");
    return PBFB_ERR_INVALID;
  }
  for (int64_t i = 0; i < 3 * (int64_t)nv; ++i)
    if (!std::isfinite(xyz[i])) {
      set_error("mesh_create: non-finite coordinate");
      return PBFB_ERR_INVALID;
    }
  for (int64_t i = 0; i < 4 * nt; ++i)
    if (tets[i] < 0 || tets[i] >= nv) {
      set_error("mesh_create: tet vertex id out of range");
      return PBFB_ERR_INVALID;
    }
  if (region) {
    int64_t cnt[2] = {0, 0};
    for (int64_t t = 0; t < nt; ++t) {
      if (region[t] != 0 && region[t] != 1) {
        set_error("mesh_create: tet region must be 0 (Omega_m) or 1 (Omega_i)");
        return PBFB_ERR_INVALID;
      }
      cnt[region[t]]++;
    }
    if (!cnt[0] || !cnt[1]) {
      set_error("mesh_create: both Omega_m and Omega_i need tets");
      return PBFB_ERR_INVALID;
    }
  }
  for (int i = 0; i < 3 * ngm; ++i)
    if (gm[i] < 0 || gm[i] >= nv) {
      set_error("mesh_create: Gamma_m vertex id out of range");
      return PBFB_ERR_INVALID;
    }
  for (int i = 0; i < 3 * ngs; ++i)
    if (gs[i] < 0 || gs[i] >= nv) {
      set_error("mesh_create: Gamma_s vertex id out of range");
      return PBFB_ERR_INVALID;
    }
  // boundary faces of the tets: faces used once, with the opposite vertex for orientation.
  // Faces are bucketed by their smallest vertex and sorted by the other two within a bucket.
  std::vector<std::array<int, 3>> fv(4 * (size_t)nt);  // sorted vertex triple of face 4 t + k
  std::vector<int> fkey(4 * (size_t)nt), fidx(4 * (size_t)nt);
  for (int64_t t = 0; t < nt; ++t) {
    const int* T = tets + 4 * t;
    double e[3][3];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) e[k][d] = xyz[3 * T[k + 1] + d] - xyz[3 * T[0] + d];
    double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                 e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    double L2 = 0.0;
    for (int k = 0; k < 3; ++k) L2 = std::max(L2, e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2]);
    if (!(std::fabs(det) > 1e-12 * L2 * std::sqrt(L2))) {
      set_error("mesh_create: degenerate tetrahedron %lld", (long long)t);
      return PBFB_ERR_INVALID;
    }
    for (int k = 0; k < 4; ++k) {
      std::array<int, 3> f;
      int q = 0;
      for (int a = 0; a < 4; ++a)
        if (a != k) f[q++] = T[a];
      std::sort(f.begin(), f.end());
      fv[4 * t + k] = f;
      fkey[4 * t + k] = f[0];
      fidx[4 * t + k] = (int)(4 * t + k);
    }
  }
  std::vector<int> fptr, ford;
  bucket(fkey, fidx, nv, fptr, ford);
  auto face_less = [&](int x, int y) { return fv[x] < fv[y]; };
  for (int v = 0; v < nv; ++v) std::sort(ford.begin() + fptr[v], ford.begin() + fptr[v + 1], face_less);
  // per sorted face position: multiplicity of its triple (1 boundary, 2 interior)
  std::vector<int> fcount(ford.size(), 0);
  size_t nb = 0, nif = 0;
  for (size_t a = 0; a < ford.size();) {
    size_t b = a + 1;
    while (b < ford.size() && fv[ford[b]] == fv[ford[a]]) ++b;
    if (b - a > 2) {
      set_error("mesh_create: a face is shared by more than two tets");
      return PBFB_ERR_INVALID;
    }
    if (b - a == 1) nb++;
    if (b - a == 2 && region && region[ford[a] / 4] != region[ford[a + 1] / 4]) nif++;
    for (size_t c = a; c < b; ++c) fcount[c] = (int)(b - a);
    a = b;
  }
  if (!region && nb != (size_t)ngm + (size_t)ngs) {
    set_error("mesh_create: %zu boundary faces but %d + %d surface triangles", nb, ngm, ngs);
    return PBFB_ERR_INVALID;
  }
  if (region && (nb != (size_t)ngs || nif != (size_t)ngm)) {
    set_error("mesh_create: %zu boundary faces and %zu Omega_m/Omega_i faces but %d Gamma_s and %d Gamma_m "
              "triangles", nb, nif, ngs, ngm);
    return PBFB_ERR_INVALID;
  }
  // position in ford of the boundary face with this sorted triple, or -1
  auto find_face = [&](const std::array<int, 3>& f) -> long long {
    auto b = ford.begin() + fptr[f[0]], e = ford.begin() + fptr[f[0] + 1];
    auto it = std::lower_bound(b, e, f, [&](int x, const std::array<int, 3>& y) { return fv[x] < y; });
    if (it == e || fv[*it] != f) return -1;
    return (long long)(it - ford.begin());
  };
  std::vector<char> onm(nv, 0), ons(nv, 0);
  for (int surf = 0; surf < 2; ++surf) {
    const int* tri = surf == 0 ? gm : gs;
    int ntri = surf == 0 ? ngm : ngs;
    std::map<std::pair<int, int>, int> dedges;
    for (int t = 0; t < ntri; ++t) {
      const int* F = tri + 3 * t;
      if (F[0] == F[1] || F[1] == F[2] || F[0] == F[2]) {
        set_error("mesh_create: repeated vertex in a surface triangle");
        return PBFB_ERR_INVALID;
      }
      std::array<int, 3> f = {F[0], F[1], F[2]};
      std::sort(f.begin(), f.end());
      const long long pos = find_face(f);
      const bool interface = region && surf == 0;  // Gamma_m between the regions
      if (interface) {
        if (pos < 0 || fcount[pos] != 2 || region[ford[pos] / 4] == region[ford[pos + 1] / 4]) {
          set_error("mesh_create: Gamma_m triangle %d is not a face between Omega_m and Omega_i tets", t);
          return PBFB_ERR_INVALID;
        }
      } else if (pos < 0 || fcount[pos] != 1) {
        set_error("mesh_create: surface triangle %d of %s is not a boundary face of the tets", t,
                  surf == 0 ? "Gamma_m" : "Gamma_s");
        return PBFB_ERR_INVALID;
      }
      fcount[pos] = 3;  // claimed
      // orientation: the opposite tet vertex lies on the positive side for Gamma_m (of the
      // Omega_i tet for an interface), on the negative side for Gamma_s
      const int fid = interface && region[ford[pos] / 4] != 1 ? ford[pos + 1] : ford[pos];
      int o = tets[fid];
      double a[3], b[3], c[3];
      for (int d = 0; d < 3; ++d) {
        a[d] = xyz[3 * F[1] + d] - xyz[3 * F[0] + d];
        b[d] = xyz[3 * F[2] + d] - xyz[3 * F[0] + d];
        c[d] = xyz[3 * o + d] - xyz[3 * F[0] + d];
      }
      double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      double side = n[0] * c[0] + n[1] * c[1] + n[2] * c[2];
      if ((surf == 0 && !(side > 0)) || (surf == 1 && !(side < 0))) {
        set_error("mesh_create: %s triangle %d has the wrong orientation", surf == 0 ? "Gamma_m" : "Gamma_s", t);
        return PBFB_ERR_INVALID;
      }
      for (int k = 0; k < 3; ++k) {
        auto key = std::make_pair(F[k], F[(k + 1) % 3]);
        if (++dedges[key] > 1) {
          set_error("mesh_create: surface is not consistently oriented / manifold");
          return PBFB_ERR_INVALID;
        }
        (surf == 0 ? onm : ons)[F[k]] = 1;
      }
    }
    for (auto& kv : dedges)
      if (!dedges.count(std::make_pair(kv.first.second, kv.first.first))) {
        set_error("mesh_create: %s is not closed", surf == 0 ? "Gamma_m" : "Gamma_s");
        return PBFB_ERR_INVALID;
      }
  }
  for (int v = 0; v < nv; ++v)
    if (onm[v] && ons[v]) {
      set_error("mesh_create: Gamma_m and Gamma_s share vertex %d", v);
      return PBFB_ERR_INVALID;
    }
  return PBFB_OK;
}

// Uniform grid over the bounding boxes of the Omega_m tets (about four tets per cell), each cell
// listing, in ascending order, the tets whose box meets it: a point's candidates are its cell's.
static void build_charge_grid(Mesh* m, const std::vector<int>& tm) {
  const int64_t nt = (int64_t)tm.size() / 4;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t k = 0; k < 4 * nt; ++k)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], m->grid_xyz[3 * (size_t)tm[k] + d]);
      hi[d] = std::max(hi[d], m->grid_xyz[3 * (size_t)tm[k] + d]);
    }
  double vol = 1.0;
  for (int d = 0; d < 3; ++d) vol *= std::max(hi[d] - lo[d], 1e-12);
  double h = std::cbrt(vol / std::max<int64_t>(1, nt / 4));
  int dim[3];
  for (int d = 0; d < 3; ++d) dim[d] = std::max(1, std::min(1024, (int)std::ceil((hi[d] - lo[d]) / h)));
  for (int d = 0; d < 3; ++d) {
    m->cell_lo[d] = lo[d];
    m->cell_dim[d] = dim[d];
  }
  m->cell_h = h;
  auto cell_range = [&](int64_t t, int* c0, int* c1) {
    for (int d = 0; d < 3; ++d) {
      double a = 1e300, b = -1e300;
      for (int v = 0; v < 4; ++v) {
        a = std::min(a, m->grid_xyz[3 * (size_t)tm[4 * t + v] + d]);
        b = std::max(b, m->grid_xyz[3 * (size_t)tm[4 * t + v] + d]);
      }
      c0[d] = std::max(0, std::min(dim[d] - 1, (int)std::floor((a - lo[d]) / h)));
      c1[d] = std::max(0, std::min(dim[d] - 1, (int)std::floor((b - lo[d]) / h)));
    }
  };
  const size_t ncell = (size_t)dim[0] * dim[1] * dim[2];
  m->cell_ptr.assign(ncell + 1, 0);
  int c0[3], c1[3];
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int> pos;
    if (pass == 1) {
      for (size_t c = 0; c < ncell; ++c) m->cell_ptr[c + 1] += m->cell_ptr[c];
      m->cell_tet.assign(m->cell_ptr[ncell], 0);
      pos.assign(m->cell_ptr.begin(), m->cell_ptr.end() - 1);
    }
    for (int64_t t = 0; t < nt; ++t) {
      cell_range(t, c0, c1);
      for (int i = c0[0]; i <= c1[0]; ++i)
        for (int j = c0[1]; j <= c1[1]; ++j)
          for (int k = c0[2]; k <= c1[2]; ++k) {
            const size_t c = ((size_t)i * dim[1] + j) * dim[2] + k;
            if (pass == 0)
              m->cell_ptr[c + 1]++;
            else
              m->cell_tet[pos[c]++] = (int)t;
          }
    }
  }
}

int point_load(Mesh* m, const double* q_xyz, const double* z, int nq, std::vector<double>& rho) {
  rho.assign(m->nv, 0.0);
  const std::vector<int>& tm = m->tets_m_h;
  const std::vector<double>& X = m->grid_xyz;
  for (int k = 0; k < nq; ++k) {
    const double* x = q_xyz + 3 * (size_t)k;
    // the cell, clamped like the tets' boxes (a point outside every box meets no tet there)
    int c[3];
    bool finite = true;
    for (int d = 0; d < 3; ++d) {
      const double f = std::floor((x[d] - m->cell_lo[d]) / m->cell_h);
      if (!std::isfinite(f)) finite = false;
      c[d] = finite ? (int)std::max(0.0, std::min((double)(m->cell_dim[d] - 1), f)) : 0;
    }
    int found = -1;
    double lam[4] = {0, 0, 0, 0};
    if (finite) {
      const size_t cell = ((size_t)c[0] * m->cell_dim[1] + c[1]) * m->cell_dim[2] + c[2];
      for (int q = m->cell_ptr[cell]; q < m->cell_ptr[cell + 1] && found < 0; ++q) {
        const int t = m->cell_tet[q];
        const int* T = &tm[4 * (size_t)t];
        // barycentric coordinates by Cramer's rule on the edge matrix E (columns x_a - x_0)
        double e[3][3], r[3];
        for (int d = 0; d < 3; ++d) {
          for (int a = 0; a < 3; ++a) e[d][a] = X[3 * (size_t)T[a + 1] + d] - X[3 * (size_t)T[0] + d];
          r[d] = x[d] - X[3 * (size_t)T[0] + d];
        }
        auto det3 = [](double a[3][3]) {
          return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                 a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
        };
        const double det = det3(e);
        double l[4];
        for (int a = 0; a < 3; ++a) {
          double ea[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) ea[i][j] = j == a ? r[i] : e[i][j];
          l[a + 1] = det3(ea) / det;
        }
        l[0] = 1.0 - l[1] - l[2] - l[3];
        if (std::min(std::min(l[0], l[1]), std::min(l[2], l[3])) >= -1e-12) {
          found = t;
          for (int a = 0; a < 4; ++a) lam[a] = l[a];
        }
      }
    }
    if (found < 0) {
      set_error("charges_set: charge %d lies in no tet of Omega_m", k);
      return PBFB_ERR_INVALID;
    }
    for (int a = 0; a < 4; ++a) rho[tm[4 * (size_t)found + a]] += z[k] * lam[a];
  }
  return PBFB_OK;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int mesh_create(const double* xyz, int nv, const int* tets, int64_t nt, const int* gm, int ngm, const int* gs,
                int ngs, cudaStream_t stream, Mesh** out, const int* region) {
  auto tc = std::chrono::steady_clock::now();
  PB_TRY(validate(xyz, nv, tets, nt, gm, ngm, gs, ngs, region));
  // tets of Omega_i (all of a shell mesh) and of Omega_m, AoS, in input order
  std::vector<int> ti_h, tm_h;
  if (region) {
    for (int64_t t = 0; t < nt; ++t) {
      std::vector<int>& dst = region[t] ? ti_h : tm_h;
      dst.insert(dst.end(), tets + 4 * t, tets + 4 * t + 4);
    }
  }
  const int* ti = region ? ti_h.data() : tets;
  const int64_t nti = region ? (int64_t)ti_h.size() / 4 : nt;
  const int64_t ntm = (int64_t)tm_h.size() / 4;
  const double t_validate = ms_since(tc);
  tc = std::chrono::steady_clock::now();
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("no CUDA device");
    return PBFB_ERR_CUDA;
  }
  PB_TRY(init_quadrature());
  PB_TRY(init_dense_attributes());
  Mesh* m = new Mesh();
  int st = PBFB_OK;
  auto fail = [&](int s) {
    delete m;
    return s;
  };
  cudaGetDevice(&m->dev);
  m->stream = stream;
  m->nv = nv;
  m->nt = nti;
  m->nt_m = ntm;
  m->full = region != nullptr;
  std::vector<double> xyz_h(xyz, xyz + 3 * (size_t)nv);
  {
    std::vector<double> soa(3 * (size_t)nv);
    for (int v = 0; v < nv; ++v)
      for (int d = 0; d < 3; ++d) soa[(size_t)d * nv + v] = xyz[3 * (size_t)v + d];
    if ((st = m->xyz.upload(soa.data(), soa.size(), stream))) return fail(st);
    for (int r = 0; r < (ntm ? 2 : 1); ++r) {
      const int* src = r == 0 ? ti : tm_h.data();
      const int64_t cnt = r == 0 ? nti : ntm;
      std::vector<int> tsoa(4 * (size_t)cnt);
      for (int64_t t = 0; t < cnt; ++t)
        for (int a = 0; a < 4; ++a) tsoa[(size_t)a * cnt + t] = src[4 * t + a];
      if ((st = (r == 0 ? m->tets : m->tets_m).upload(tsoa.data(), tsoa.size(), stream))) return fail(st);
    }
  }
  std::vector<int> gmv(gm, gm + 3 * (size_t)ngm), gsv(gs, gs + 3 * (size_t)ngs);
  {
    // the two surfaces are independent: Gamma_s on a second host thread (its own error text)
    int st_s = PBFB_OK;
    std::string err_s;
    std::thread th([&] {
      cudaSetDevice(m->dev);
      st_s = build_surface(m, &m->ss, gsv, xyz_h);
      if (st_s != PBFB_OK) err_s = last_error();
    });
    st = build_surface(m, &m->sm, gmv, xyz_h);
    th.join();
    if (st) return fail(st);
    if (st_s) {
      set_error("%s", err_s.c_str());
      return fail(st_s);
    }
  }
  Surface& sm = m->sm;
  Surface& ss = m->ss;
  m->setup_ms[0] = t_validate;
  m->setup_ms[1] = ms_since(tc);
  tc = std::chrono::steady_clock::now();
  sm.col0 = nv;
  ss.col0 = nv + sm.nv;
  m->n = nv + sm.nv + ss.nv;
  // ---- sparse-part pattern of the coupled operator
  std::vector<int64_t> keys;
  keys.reserve(16 * (size_t)nt + 4 * (size_t)(sm.cnnz + ss.cnnz));
  for (int r = 0; r < 2; ++r) {
    const int* tt = r == 0 ? ti : tm_h.data();
    const int64_t cnt = r == 0 ? nti : ntm;
    for (int64_t t = 0; t < cnt; ++t)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) keys.push_back(key2(tt[4 * t + a], tt[4 * t + b]));
  }
  // mass pattern (vertices sharing a triangle) for the FEM coupling entries
  auto mass_pairs = [](const Surface& s, std::vector<std::pair<int, int>>& mp) {
    for (int t = 0; t < s.nt; ++t)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) mp.push_back({s.tri_h[3 * t + a], s.tri_h[3 * t + b]});
    std::sort(mp.begin(), mp.end());
    mp.erase(std::unique(mp.begin(), mp.end()), mp.end());
  };
  // (an interior Gamma_m couples nothing: its lam_m rows are the identity)
  std::vector<std::pair<int, int>> mpm, mps;
  if (!m->full) mass_pairs(sm, mpm);
  mass_pairs(ss, mps);
  for (auto& e : mpm) keys.push_back(key2(sm.vmap_h[e.first], sm.col0 + e.second));
  for (auto& e : mps) keys.push_back(key2(ss.vmap_h[e.first], ss.col0 + e.second));
  for (const Surface* s : {&sm, &ss}) {
    if (m->full && s == &sm) {
      for (int i = 0; i < s->nv; ++i) keys.push_back(key2(s->col0 + i, s->col0 + i));
      continue;
    }
    for (int i = 0; i < s->nv; ++i)
      for (int k = s->c_ptr_h[i]; k < s->c_ptr_h[i + 1]; ++k) {
        int j = s->c_col_h[k];
        keys.push_back(key2(s->col0 + i, s->vmap_h[j]));
        keys.push_back(key2(s->col0 + i, s->col0 + j));
      }
  }
  {
    // rows by counting sort, then sorted unique columns within each row
    std::vector<int> rk(keys.size()), ck(keys.size());
    for (size_t k = 0; k < keys.size(); ++k) {
      rk[k] = (int)(keys[k] >> 32);
      ck[k] = (int)(keys[k] & 0xffffffff);
    }
    std::vector<int>().swap(m->s_col_h);
    std::vector<int64_t>().swap(keys);
    std::vector<int> rptr, cols;
    bucket(rk, ck, m->n, rptr, cols);
    m->s_ptr_h.assign(m->n + 1, 0);
    size_t w = 0;
    std::vector<char> seen(m->n, 0);
    for (int r = 0; r < m->n; ++r) {
      // distinct columns of the row (a marker per column), then sorted in place
      const size_t w0 = w;
      for (int q = rptr[r]; q < rptr[r + 1]; ++q) {
        const int c = cols[q];
        if (!seen[c]) {
          seen[c] = 1;
          cols[w++] = c;
        }
      }
      std::sort(cols.begin() + w0, cols.begin() + w);
      for (size_t q = w0; q < w; ++q) seen[cols[q]] = 0;
      m->s_ptr_h[r + 1] = (int)w;
    }
    cols.resize(w);
    m->s_col_h.swap(cols);
    m->snnz = (int)w;
  }
  m->fem_nnz = m->s_ptr_h[nv];
  auto slot = [&](int r, int c) -> int {
    auto b = m->s_col_h.begin() + m->s_ptr_h[r], e = m->s_col_h.begin() + m->s_ptr_h[r + 1];
    return (int)(std::lower_bound(b, e, c) - m->s_col_h.begin());
  };
  std::vector<int> kind(m->snnz, -1), ref(m->snnz, 0);
  DBuf<int> jm_ptr, jm_idx;  // Omega_m stiffness gather (set-up only)
  {
    // per slot: tet-local entries (k * cnt + t) of the Omega_i tets, and of the Omega_m tets
    std::vector<int> ptr, outv;
    for (int r = 0; r < (ntm ? 2 : 1); ++r) {
      const int* tt = r == 0 ? ti : tm_h.data();
      const int64_t cnt = r == 0 ? nti : ntm;
      std::vector<int> jk, jv;
      jk.reserve(16 * (size_t)cnt);
      jv.reserve(16 * (size_t)cnt);
      for (int64_t t = 0; t < cnt; ++t)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            int sl = slot(tt[4 * t + a], tt[4 * t + b]);
            kind[sl] = 0;
            jk.push_back(sl);
            jv.push_back((int)(sym10(a, b) * cnt + t));
          }
      bucket(jk, jv, m->snnz, ptr, outv);
      if ((st = (r == 0 ? m->jg_ptr : jm_ptr).upload(ptr.data(), ptr.size(), stream))) return fail(st);
      if ((st = (r == 0 ? m->jg_idx : jm_idx).upload(outv.data(), outv.size(), stream))) return fail(st);
    }
    std::vector<int> nk, nvv;
    for (int64_t t = 0; t < nti; ++t)
      for (int a = 0; a < 4; ++a) {
        nk.push_back(ti[4 * t + a]);
        nvv.push_back((int)(a * nti + t));
      }
    bucket(nk, nvv, nv, ptr, outv);
    if ((st = m->ng_ptr.upload(ptr.data(), ptr.size(), stream))) return fail(st);
    if ((st = m->ng_idx.upload(outv.data(), outv.size(), stream))) return fail(st);
  }
  auto cslot = [](const Surface& s, int i, int j) -> int {
    auto b = s.c_col_h.begin() + s.c_ptr_h[i], e = s.c_col_h.begin() + s.c_ptr_h[i + 1];
    return (int)(std::lower_bound(b, e, j) - s.c_col_h.begin());
  };
  for (auto& e : mpm) {
    int sl = slot(sm.vmap_h[e.first], sm.col0 + e.second);
    kind[sl] = 1;
    ref[sl] = cslot(sm, e.first, e.second);
  }
  for (auto& e : mps) {
    int sl = slot(ss.vmap_h[e.first], ss.col0 + e.second);
    kind[sl] = 2;
    ref[sl] = cslot(ss, e.first, e.second);
  }
  {
    // Robin term of the block preconditioner: u-u slots of Gamma_s vertex pairs sharing a triangle
    std::vector<int> rs, rr;
    for (auto& e : mps) {
      rs.push_back(slot(ss.vmap_h[e.first], ss.vmap_h[e.second]));
      rr.push_back(cslot(ss, e.first, e.second));
    }
    m->nrobin = (int)rs.size();
    if ((st = m->robin_slot.upload(rs.data(), rs.size(), stream))) return fail(st);
    if ((st = m->robin_ref.upload(rr.data(), rr.size(), stream))) return fail(st);
    double area = 0.0;
    for (int t = 0; t < ss.nt; ++t) {
      const int* T = &ss.tri_h[3 * t];
      double a[3], b[3];
      for (int d = 0; d < 3; ++d) {
        a[d] = xyz_h[3 * (size_t)ss.vmap_h[T[1]] + d] - xyz_h[3 * (size_t)ss.vmap_h[T[0]] + d];
        b[d] = xyz_h[3 * (size_t)ss.vmap_h[T[2]] + d] - xyz_h[3 * (size_t)ss.vmap_h[T[0]] + d];
      }
      double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
      area += 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    m->gs_radius = std::sqrt(area / (4.0 * M_PI));
  }
  if (!m->full) {
    // Gamma_m's triangles (as stored: normal out of the solute) for the charges' winding numbers
    m->gm_tri_xyz.resize(9 * (size_t)sm.nt);
    for (int t = 0; t < sm.nt; ++t)
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d)
          m->gm_tri_xyz[9 * (size_t)t + 3 * a + d] = xyz_h[3 * (size_t)sm.vmap_h[sm.tri_h[3 * t + a]] + d];
  }
  for (int si = 0; si < 2; ++si) {
    const Surface& s = si == 0 ? sm : ss;
    if (m->full && si == 0) {
      for (int i = 0; i < s.nv; ++i) kind[slot(s.col0 + i, s.col0 + i)] = 7;
      continue;
    }
    for (int i = 0; i < s.nv; ++i)
      for (int k = s.c_ptr_h[i]; k < s.c_ptr_h[i + 1]; ++k) {
        int j = s.c_col_h[k];
        int a = slot(s.col0 + i, s.vmap_h[j]);
        int b = slot(s.col0 + i, s.col0 + j);
        kind[a] = si == 0 ? 3 : 5;
        ref[a] = k;
        kind[b] = si == 0 ? 4 : 6;
        ref[b] = k;
      }
  }
  for (int k = 0; k < m->snnz; ++k)
    if (kind[k] < 0) {
      set_error("internal: unassigned operator slot");
      return fail(PBFB_ERR_STATE);
    }
  if ((st = m->s_ptr.upload(m->s_ptr_h.data(), m->s_ptr_h.size(), stream))) return fail(st);
  if ((st = m->s_col.upload(m->s_col_h.data(), m->s_col_h.size(), stream))) return fail(st);
  if ((st = m->s_kind.upload(kind.data(), kind.size(), stream))) return fail(st);
  if ((st = m->s_ref.upload(ref.data(), ref.size(), stream))) return fail(st);
  if ((st = m->s_val.alloc(m->snnz))) return fail(st);
  if ((st = m->s_base.alloc(m->snnz))) return fail(st);
  if ((st = m->a1.alloc(m->snnz))) return fail(st);
  if ((st = m->vol.alloc(nti))) return fail(st);
  if ((st = m->tloc.alloc(14 * (size_t)nti))) return fail(st);
  if ((st = m->red.alloc((size_t)152 * 7 * 64 + 1024))) return fail(st);
  if ((st = m->scal.alloc(8192))) return fail(st);
  if ((st = m->red2.alloc(9 * (size_t)std::max(sm.npair, ss.npair)))) return fail(st);
  if (cudaMallocHost((void**)&m->pinned, 4096 * sizeof(double)) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    return fail(PBFB_ERR_OOM);
  }
  m->setup_ms[2] = ms_since(tc);
  tc = std::chrono::steady_clock::now();
  // ---- device geometry and constant operator parts
  if ((st = launch_tet_volumes(m, m->tets.p, m->nt, m->vol.p))) return fail(st);
  if ((st = launch_stiffness_local(m, m->tets.p, m->nt, m->vol.p, m->tloc.p))) return fail(st);
  if ((st = launch_gather(m, m->snnz, m->jg_ptr.p, m->jg_idx.p, m->tloc.p, nullptr, 1.0, m->a1.p))) return fail(st);
  DBuf<double> locm;
  if (m->full) {
    if ((st = m->vol_m.alloc(ntm)) || (st = m->a1m.alloc(m->snnz)) || (st = locm.alloc(10 * (size_t)ntm)))
      return fail(st);
    if ((st = launch_tet_volumes(m, m->tets_m.p, ntm, m->vol_m.p))) return fail(st);
    if ((st = launch_stiffness_local(m, m->tets_m.p, ntm, m->vol_m.p, locm.p))) return fail(st);
    if ((st = launch_gather(m, m->snnz, jm_ptr.p, jm_idx.p, locm.p, nullptr, 1.0, m->a1m.p))) return fail(st);
    m->grid_xyz.swap(xyz_h);
    build_charge_grid(m, tm_h);
    m->tets_m_h.swap(tm_h);
  }
  if ((st = launch_surface_geometry(m, &sm))) return fail(st);
  if ((st = launch_surface_geometry(m, &ss))) return fail(st);
  if ((st = launch_pair_corrections(m, &sm, 0.0))) return fail(st);
  sm.kappa = 0.0;
  sm.built = true;
  if (cudaStreamSynchronize(stream) != cudaSuccess) {
    set_error("mesh_create: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(PBFB_ERR_CUDA);
  }
  m->setup_ms[3] = ms_since(tc);
  *out = m;
  return PBFB_OK;
}

// Generalised winding number of a closed triangulated surface at points q (n of them):
// w(x) = (1/4 pi) sum_tau Omega_tau(x), with the signed solid angle of each triangle from the formula
// of Van Oosterom and Strackee (1983),
//   tan(Omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| + (b.c)|a| + (c.a)|b|),  a, b, c = corners - x.
// With the normals pointing out of the enclosed region, w = 1 inside, 0 outside and 1/2 on the
// surface.  A point on a triangle (a corner, or coplanar to 1e-12 relative with the formula's
// denominator not positive, i.e. within the triangle) makes that triangle's solid angle +-2 pi by
// the sign of a rounded zero; such points are reported as on the surface, w = 1/2.
// tri9: 9 coordinates per triangle.  Host threads over the points.
void winding_numbers(const double* tri9, size_t nt, const double* q, int nq, double* w) {
  auto work = [&](int k0, int k1) {
    for (int k = k0; k < k1; ++k) {
      const double x = q[3 * k], y = q[3 * k + 1], z = q[3 * k + 2];
      double sum = 0.0;
      bool on = false;
      for (size_t t = 0; t < nt; ++t) {
        const double* P = tri9 + 9 * t;
        const double a0 = P[0] - x, a1 = P[1] - y, a2 = P[2] - z;
        const double b0 = P[3] - x, b1 = P[4] - y, b2 = P[5] - z;
        const double c0 = P[6] - x, c1 = P[7] - y, c2 = P[8] - z;
        const double la = std::sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        const double lb = std::sqrt(b0 * b0 + b1 * b1 + b2 * b2);
        const double lc = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        const double det = a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
        const double den = la * lb * lc + (a0 * b0 + a1 * b1 + a2 * b2) * lc + (b0 * c0 + b1 * c1 + b2 * c2) * la +
                           (c0 * a0 + c1 * a1 + c2 * a2) * lb;
        const double s3 = la * lb * lc;
        if (s3 == 0.0 || (std::fabs(det) <= 1e-12 * s3 && den <= 0.0)) on = true;
        sum += 2.0 * std::atan2(det, den);
      }
      w[k] = on ? 0.5 : sum / (4.0 * M_PI);
    }
  };
  const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (nth == 1 || nq < 2 || (double)nq * (double)nt < 2e5) {
    work(0, nq);
    return;
  }
  const int nuse = std::min(nth, nq);
  std::vector<std::thread> th;
  for (int i = 0; i < nuse; ++i)
    th.emplace_back(work, (int)((int64_t)nq * i / nuse), (int)((int64_t)nq * (i + 1) / nuse));
  for (auto& t : th) t.join();
}

// Every charge strictly inside the closed surface (the charges of the three-region model lie in
// Omega_m, Sec. 2.1): winding number above 3/4.  w (may be null) receives the winding numbers.
int check_charges_inside(const double* tri9, size_t nt, const double* q, int nq, double* w_out) {
  std::vector<double> w(nq, 0.0);
  winding_numbers(tri9, nt, q, nq, w.data());
  if (w_out) std::copy(w.begin(), w.end(), w_out);
  for (int k = 0; k < nq; ++k)
    if (!(w[k] > 0.75)) {
      set_error("charge %d at (%g, %g, %g) is not strictly inside Gamma_m (winding number %.3f)", k, q[3 * k],
                q[3 * k + 1], q[3 * k + 2], w[k]);
      return PBFB_ERR_INVALID;
    }
  return PBFB_OK;
}

int charges_inside_gamma_m(const Mesh* m, const double* q, int nq) {
  const size_t nt = m->gm_tri_xyz.size() / 9;
  if (nt == 0) return PBFB_OK;
  return check_charges_inside(m->gm_tri_xyz.data(), nt, q, nq, nullptr);
}

}  // namespace pbfb

// ==================================================================== C ABI (host only)

extern "C" int pbfb_check_charges(const double* xyz, int32_t n_v, const int32_t* gm_tris, int32_t n_gm,
                                  const double* q_xyz, int32_t n_q, double* winding_out) {
  pbfb::set_error("");
  if (!xyz || !gm_tris || !q_xyz || n_v < 3 || n_gm < 4 || n_q < 1) {
    pbfb::set_error("check_charges: bad argument");
    return PBFB_ERR_INVALID;
  }
  std::vector<double> tri9(9 * (size_t)n_gm);
  for (int32_t t = 0; t < n_gm; ++t)
    for (int a = 0; a < 3; ++a) {
      const int32_t v = gm_tris[3 * (size_t)t + a];
      if (v < 0 || v >= n_v) {
        pbfb::set_error("check_charges: vertex id %d out of range", v);
        return PBFB_ERR_INVALID;
      }
      for (int d = 0; d < 3; ++d) tri9[9 * (size_t)t + 3 * a + d] = xyz[3 * (size_t)v + d];
    }
  for (int32_t k = 0; k < 3 * n_q; ++k)
    if (!std::isfinite(q_xyz[k])) {
      pbfb::set_error("check_charges: non-finite position");
      return PBFB_ERR_INVALID;
    }
  return pbfb::check_charges_inside(tri9.data(), (size_t)n_gm, q_xyz, n_q, winding_out);
}
