// Request server and batch solve (include/pbfb.h: pbfb_server_*, pbfb_solve_batch).
//
// Serving form of the solver: requests (mesh, charges, parameters) are queued as they arrive,
// admitted in arrival order while their estimated device memory fits the budget, and solved by a
// pool of worker threads, each with its own non-blocking CUDA stream, so the set-up (host) and
// GPU work of different requests overlap.  Every request is solved on its own mesh, stream and
// buffers with deterministic kernels, so its result does not depend on what else is in flight.
// Meshes solved concurrently use the multi-kernel inner PCG (no grid-wide barrier, which could
// not be guaranteed co-resident when several run at once).  Up to `cached_meshes` meshes stay on
// the device after their request; a later request with the same geometry (compared exactly)
// reuses one instead of building it again.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "pbfb_internal.cuh"

namespace pbfb {

// Device bytes a solve of this size holds (buffers of mesh_create, the solve workspace, GMRES with
// the flexible basis, the dense preconditioner blocks), with a 25% margin.
size_t estimate_bytes(int64_t nv, int64_t nt, int64_t ngm, int64_t ngs, int restart) {
  const double nm = ngm / 2.0 + 2, ns = ngs / 2.0 + 2;  // closed triangulations: V = F/2 + 2
  const double n = nv + nm + ns;
  const double nnz_fem = 16.0 * nv + 20.0 * (nm + ns);
  double b = 0;
  b += nt * (4 * 4 + 8 + 14 * 8 + 12 * 8 + 16 * 4);              // tets, volume, tet-local, one omega, gather idx
  b += nv * (3 * 8 + 4 * 4 + 10 * 8);                             // coordinates, gather pointers, vectors
  b += nnz_fem * (4 + 8 * 4 + 4 * 2);                             // CSR, values, base, a1, pval, descriptors
  for (double nqs : {6.0 * ngm, 6.0 * ngs}) {
    const double npair = nqs / 6.0 * 60.0;                        // special pairs (touching + near)
    b += nqs * (3 * 8 + 8 + 16 + 32 + 7 * 8 + 96) + (double)far_splits_max((int64_t)nqs) * nqs * 8;
    b += npair * (9 * 8 * 4 + 16 * 4) + 40.0 * nqs / 6.0 * (4 + 8 * 3);
    b += nqs * 140.0 * 8;                                         // mutual float-float partial rows
    b += nqs * 500.0;                                             // treecode: tree-order records, proxies, partials
  }
  b += (2.0 * restart + 1 + 16) * n * 8;                          // Krylov V, Z, work vectors
  // dense single-layer inverses of the block preconditioner and their build scratch
  for (double nsv : {nm, ns})
    if (nsv <= DENSE_V_MAX) b += (double)dense_bytes((int)nsv);
  const double nbig = std::min(std::max(nm, ns), (double)DENSE_V_MAX);
  b += (double)dense_work_bytes((int)nbig, (int)(2 * nbig));
  return (size_t)(1.25 * b) + (64u << 20);
}

namespace {

struct Request {
  int64_t id = 0;
  std::vector<double> xyz, qxyz, qz;
  std::vector<int> tets, gm, gs;
  std::vector<int> region;  // per tet 0 (Omega_m) / 1 (Omega_i); empty for a shell mesh
  double eps_in = 0, eps_out = 0, kappa = 0, T = 0;
  pbfb_newton_opts opts;
  size_t bytes = 0;
  uint64_t hash = 0;  // of the geometry (coordinates, tets, both surfaces, tet regions)
  double t_submit = 0;
};

// A mesh kept on the device between requests with the same geometry (its topology, geometry,
// near-field corrections, dense single-layer inverses and solve workspace stay resident).
struct Cached {
  uint64_t hash = 0;
  std::vector<double> xyz;
  std::vector<int> tets, gm, gs, region;
  Mesh* m = nullptr;
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

// FNV-1a over the bytes of the geometry arrays
uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t geometry_hash(const Request& r) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, r.xyz.data(), r.xyz.size() * sizeof(double));
  h = fnv(h, r.tets.data(), r.tets.size() * sizeof(int));
  h = fnv(h, r.gm.data(), r.gm.size() * sizeof(int));
  h = fnv(h, r.region.data(), r.region.size() * sizeof(int));
  return fnv(h, r.gs.data(), r.gs.size() * sizeof(int));
}

bool same_geometry(const Request& r, const Cached& c) {
  return r.xyz == c.xyz && r.tets == c.tets && r.gm == c.gm && r.gs == c.gs && r.region == c.region;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Server {
  int dev = 0;
  size_t budget = 0, in_use = 0, peak = 0;
  int nworkers = 0;
  int max_cached = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::deque<pbfb_response> done;
  std::vector<std::thread> workers;
  std::vector<Cached*> cache;   // in_use counts every cached mesh, busy or idle
  uint64_t tick = 0;
  bool stop = false;
  int64_t submitted = 0, completed = 0, hits = 0;

  // an idle cached mesh of exactly this geometry, or null (under mu): the hash selects the
  // candidates and the arrays are compared in full, so that a hash collision is never taken for
  // a hit (admission would then not account for the fresh mesh the request needs)
  Cached* find_idle(const Request* r) {
    for (Cached* c : cache)
      if (!c->busy && c->hash == r->hash && same_geometry(*r, *c)) return c;
    return nullptr;
  }

  // drop idle cached meshes, least recently used first, until `need` more bytes fit (under mu);
  // the meshes are destroyed by the caller after releasing the lock
  void evict_for(size_t need, std::vector<Mesh*>& dead) {
    while (in_use > 0 && in_use + need > budget) {
      Cached* lru = nullptr;
      for (Cached* c : cache)
        if (!c->busy && (!lru || c->last_use < lru->last_use)) lru = c;
      if (!lru) return;
      cache.erase(std::find(cache.begin(), cache.end(), lru));
      in_use -= lru->bytes;
      dead.push_back(lru->m);
      delete lru;
    }
  }

  void run_worker() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    while (true) {
      Request* r = nullptr;
      Cached* hit = nullptr;
      std::vector<Mesh*> dead;
      {
        // take the head of the queue once it fits: on an idle cached mesh of its geometry (no new
        // memory), or in the budget after evicting idle cached meshes (a request alone always
        // fits); cv_work is signalled on new requests, on completions and on shutdown
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
          if (!queue.empty()) {
            Request* head = queue.front();
            hit = find_idle(head);
            if (!hit) evict_for(head->bytes, dead);
            if (hit || in_use == 0 || in_use + head->bytes <= budget) {
              r = head;
              queue.pop_front();
              if (hit) {
                hit->busy = true;
              } else {
                in_use += r->bytes;
                peak = std::max(peak, in_use);
              }
              break;
            }
          }
          cv_work.wait(lk);
        }
      }
      for (Mesh* dm : dead) mesh_destroy(dm);
      if (!r) break;
      pbfb_response resp;
      std::memset(&resp, 0, sizeof(resp));
      resp.id = r->id;
      resp.t_submit_ms = r->t_submit;
      resp.t_start_ms = now_ms();
      Mesh* m = nullptr;
      int st = PBFB_OK;
      if (hit) {
        m = hit->m;
        m->stream = s;  // the mesh is idle: its earlier work ended with a synchronisation
      } else {
        st = mesh_create(r->xyz.data(), (int)(r->xyz.size() / 3), r->tets.data(), (int64_t)(r->tets.size() / 4),
                         r->gm.data(), (int)(r->gm.size() / 3), r->gs.data(), (int)(r->gs.size() / 3), s, &m,
                         r->region.empty() ? nullptr : r->region.data());
        if (st == PBFB_OK) m->no_coop = true;
      }
      if (st == PBFB_OK) st = charges_set(m, r->qxyz.data(), r->qz.data(), (int)r->qz.size());
      if (st == PBFB_OK) st = solve_mesh(m, r->eps_in, r->eps_out, r->kappa, r->T, &r->opts, nullptr, &resp.result);
      if (st != PBFB_OK) std::strncpy(resp.error, last_error(), sizeof(resp.error) - 1);
      resp.status = st;
      resp.result.status = st;
      Mesh* drop = nullptr;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (hit) {
          hit->busy = false;
          hit->last_use = ++tick;
          ++hits;
        } else if (st == PBFB_OK && m && (int)cache.size() < max_cached) {
          Cached* c = new Cached();
          c->hash = r->hash;
          c->xyz.swap(r->xyz);
          c->tets.swap(r->tets);
          c->gm.swap(r->gm);
          c->gs.swap(r->gs);
          c->region.swap(r->region);
          c->m = m;
          c->bytes = r->bytes;
          c->last_use = ++tick;
          cache.push_back(c);
        } else {
          drop = m;
          in_use -= r->bytes;
        }
        resp.t_done_ms = now_ms();
        done.push_back(resp);
        ++completed;
      }
      if (drop) mesh_destroy(drop);
      delete r;
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (s) cudaStreamDestroy(s);
  }
};

}  // namespace pbfb

// ==================================================================== C ABI

struct pbfb_server {
  pbfb::Server* s;
};

extern "C" {

int pbfb_server_create(int device, uint64_t hbm_budget_bytes, int max_inflight, int cached_meshes,
                       pbfb_server** out) {
  pbfb::set_error("");
  if (!out || max_inflight < 1 || max_inflight > 64 || hbm_budget_bytes == 0 || cached_meshes < 0 ||
      cached_meshes > 1024) {
    pbfb::set_error("server_create: bad argument");
    return PBFB_ERR_INVALID;
  }
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    pbfb::set_error("server_create: no CUDA device %d", device);
    return PBFB_ERR_CUDA;
  }
  auto* sv = new pbfb::Server();
  sv->dev = device;
  sv->budget = hbm_budget_bytes;
  sv->nworkers = max_inflight;
  sv->max_cached = cached_meshes;
  for (int i = 0; i < max_inflight; ++i) sv->workers.emplace_back([sv] { sv->run_worker(); });
  *out = new pbfb_server{sv};
  return PBFB_OK;
}

int pbfb_server_submit(pbfb_server* h, const pbfb_request* q) {
  if (!h || !h->s || !q || !q->xyz || !q->tets || !q->gm_tris || !q->gs_tris || !q->q_xyz || !q->q_z ||
      q->n_v < 4 || q->n_t < 1 || q->n_gm < 4 || q->n_gs < 4 || q->n_q < 1) {
    pbfb::set_error("server_submit: bad request");
    return PBFB_ERR_INVALID;
  }
  pbfb::Server* sv = h->s;
  auto* r = new pbfb::Request();
  r->id = q->id;
  r->xyz.assign(q->xyz, q->xyz + 3 * (size_t)q->n_v);
  r->tets.assign(q->tets, q->tets + 4 * (size_t)q->n_t);
  r->gm.assign(q->gm_tris, q->gm_tris + 3 * (size_t)q->n_gm);
  r->gs.assign(q->gs_tris, q->gs_tris + 3 * (size_t)q->n_gs);
  if (q->tet_region) r->region.assign(q->tet_region, q->tet_region + q->n_t);
  r->qxyz.assign(q->q_xyz, q->q_xyz + 3 * (size_t)q->n_q);
  r->qz.assign(q->q_z, q->q_z + q->n_q);
  r->eps_in = q->eps_in;
  r->eps_out = q->eps_out;
  r->kappa = q->kappa;
  r->T = q->T;
  pbfb_default_opts(&r->opts);
  if (q->opts) r->opts = *q->opts;
  r->bytes = pbfb::estimate_bytes(q->n_v, q->n_t, q->n_gm, q->n_gs, r->opts.restart);
  r->hash = pbfb::geometry_hash(*r);
  r->t_submit = pbfb::now_ms();
  if (r->bytes > sv->budget) {
    pbfb::set_error("server_submit: request needs about %zu bytes, more than the budget %zu", r->bytes, sv->budget);
    delete r;
    return PBFB_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete r;
      pbfb::set_error("server_submit: server is shutting down");
      return PBFB_ERR_STATE;
    }
    sv->queue.push_back(r);
    ++sv->submitted;
  }
  sv->cv_work.notify_all();
  return PBFB_OK;
}

int pbfb_server_poll(pbfb_server* h, pbfb_response* out, int max, int timeout_us, int* n_out) {
  if (!h || !h->s || !out || max < 1 || !n_out) {
    pbfb::set_error("server_poll: bad argument");
    return PBFB_ERR_INVALID;
  }
  pbfb::Server* sv = h->s;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->done.empty() && timeout_us > 0)
    sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !sv->done.empty(); });
  int n = 0;
  while (n < max && !sv->done.empty()) {
    out[n++] = sv->done.front();
    sv->done.pop_front();
  }
  *n_out = n;
  if (n == 0 && timeout_us > 0) {
    pbfb::set_error("server_poll: no response within %d us", timeout_us);
    return PBFB_ERR_TIMEOUT;
  }
  return PBFB_OK;
}

int pbfb_server_stats(pbfb_server* h, double* stats) {
  if (!h || !h->s || !stats) {
    pbfb::set_error("server_stats: bad argument");
    return PBFB_ERR_INVALID;
  }
  pbfb::Server* sv = h->s;
  std::lock_guard<std::mutex> lk(sv->mu);
  stats[0] = (double)sv->submitted;
  stats[1] = (double)sv->completed;
  stats[2] = (double)sv->queue.size();
  stats[3] = (double)sv->in_use;
  stats[4] = (double)sv->peak;
  stats[5] = (double)sv->budget;
  stats[6] = (double)sv->hits;
  stats[7] = (double)sv->cache.size();
  return PBFB_OK;
}

int pbfb_server_destroy(pbfb_server* h) {
  if (!h) return PBFB_OK;
  pbfb::Server* sv = h->s;
  if (sv) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    for (auto* r : sv->queue) delete r;
    // the workers have finished every solve and destroyed their streams: the resident meshes
    // still name one of those streams, so they are released on the legacy stream instead
    for (auto* c : sv->cache) {
      c->m->stream = nullptr;
      pbfb::mesh_destroy(c->m);
      delete c;
    }
    delete sv;
  }
  delete h;
  return PBFB_OK;
}

int pbfb_solve_batch(pbfb_mesh* const* meshes, const pbfb_batch_params* params, int n, int max_concurrent,
                     pbfb_result* results) {
  if (!meshes || !params || !results || n < 1 || max_concurrent < 1) {
    pbfb::set_error("solve_batch: bad argument");
    return PBFB_ERR_INVALID;
  }
  std::vector<int> status(n, PBFB_OK);
  std::vector<std::string> errs(n);
  std::mutex mu;
  int next = 0;
  auto work = [&] {
    while (true) {
      int i;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (next >= n) return;
        i = next++;
      }
      pbfb::Mesh* m = pbfb_mesh_internal(meshes[i]);
      if (!m) {
        status[i] = PBFB_ERR_INVALID;
        continue;
      }
      const bool save = m->no_coop;
      m->no_coop = true;
      int st = pbfb::solve_mesh(m, params[i].eps_in, params[i].eps_out, params[i].kappa, params[i].T,
                                params[i].opts, nullptr, &results[i]);
      m->no_coop = save;
      status[i] = st;
      results[i].status = st;
      if (st) errs[i] = pbfb_last_error();
    }
  };
  std::vector<std::thread> th;
  for (int k = 0; k < std::min(n, max_concurrent); ++k) th.emplace_back(work);
  for (auto& t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (status[i]) {
      pbfb::set_error("solve_batch: instance %d: %s", i, errs[i].c_str());
      return status[i];
    }
  return PBFB_OK;
}

}  // extern "C"
