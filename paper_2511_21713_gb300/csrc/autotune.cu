// Autotuner of the launch shapes (include/pbfb.h: pbfb_autotune, pbfb_get_tuning,
// pbfb_apply_tuning).  Candidates are timed with CUDA events on the mesh's stream on the
// mesh's own surfaces and sparse pattern; the fastest is applied to the mesh.
#include <cuda_runtime.h>

#include <vector>

#include "pbfb_internal.cuh"

namespace pbfb {

namespace {

void read_tuning(const Mesh* m, pbfb_tuning* t) {
  t->nbody_targets_per_thread = m->tune_tpt;
  t->nbody_blocks_per_sm = m->tune_bps;
  t->nbody_packed = m->tune_packed;
  t->ff_blocks_per_sm = m->tune_ff_bps;
  t->ff_kernel = m->tune_ff_kernel;
  t->spmv_lanes = m->spmv_lanes;
  t->spmv_block = m->spmv_block;
  t->pcg_blocks_per_sm = m->tune_pcg_bps;
  t->pcg_lanes = m->pcg_lanes;
  t->treecode = m->tune_tree;
  t->pcg_precision = m->tune_pcg_prec;
}

bool valid_tuning(const pbfb_tuning* t) {
  auto in = [](int v, int lo, int hi) { return v == 0 || (v >= lo && v <= hi); };
  const int tp = t->nbody_targets_per_thread;
  if (!(tp == 0 || tp == 1 || tp == 2 || tp == 4 || tp == 8)) return false;
  if (!in(t->nbody_blocks_per_sm, 1, 64) || !in(t->ff_blocks_per_sm, 1, 64)) return false;
  if (t->nbody_packed < 0 || t->nbody_packed > 2 || t->ff_kernel < 0 || t->ff_kernel > 4) return false;
  if (t->nbody_packed == 1 && tp != 0 && tp < 2) return false;
  if (t->nbody_packed == 2 && tp != 4) return false;
  const int L = t->spmv_lanes, B = t->spmv_block;
  if (!(L == 0 || L == 4 || L == 8 || L == 16)) return false;
  if (!(B == 0 || B == 128 || B == 256 || B == 512)) return false;
  if (!in(t->pcg_blocks_per_sm, 1, 32)) return false;
  if (!(t->pcg_lanes == 0 || t->pcg_lanes == 1 || t->pcg_lanes == 2 || t->pcg_lanes == 4 || t->pcg_lanes == 8))
    return false;
  if (t->treecode < 0 || t->treecode > 3) return false;
  if (t->pcg_precision < 0 || t->pcg_precision > 2) return false;
  return true;
}

void write_tuning(Mesh* m, const pbfb_tuning* t) {
  m->tune_tpt = t->nbody_targets_per_thread;
  m->tune_bps = t->nbody_blocks_per_sm;
  m->tune_packed = t->nbody_packed;
  m->tune_ff_bps = t->ff_blocks_per_sm;
  m->tune_ff_kernel = t->ff_kernel;
  m->spmv_lanes = t->spmv_lanes;
  m->spmv_block = t->spmv_block;
  if (m->tune_pcg_bps != t->pcg_blocks_per_sm) m->coop_blocks = 0;  // re-derive the grid
  m->tune_pcg_bps = t->pcg_blocks_per_sm;
  m->pcg_lanes = t->pcg_lanes;
  m->tune_tree = t->treecode;
  m->tune_pcg_prec = t->pcg_precision;
}

// milliseconds per repetition of fn (one untimed run first)
template <class F>
int time_ms(Mesh* m, int reps, F fn, double* ms) {
  PB_TRY(fn());
  cudaEvent_t a, b;
  PB_CUDA(cudaEventCreate(&a));
  PB_CUDA(cudaEventCreate(&b));
  PB_CUDA(cudaEventRecord(a, m->stream));
  for (int r = 0; r < reps; ++r) PB_TRY(fn());
  PB_CUDA(cudaEventRecord(b, m->stream));
  PB_CUDA(cudaEventSynchronize(b));
  float t = 0.f;
  PB_CUDA(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return PBFB_OK;
}

}  // namespace

int autotune(Mesh* m, int reps, pbfb_tuning* best_out, double* ms_out) {
  DBuf<double> x, y;
  PB_TRY(x.alloc(m->n));
  PB_TRY(y.alloc(m->n));
  {
    std::vector<double> h(m->n);
    for (int i = 0; i < m->n; ++i) h[i] = 1.0 + 0.001 * (i % 97);
    PB_CUDA(cudaMemcpyAsync(x.p, h.data(), m->n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    PB_CUDA(cudaStreamSynchronize(m->stream));
  }
  pbfb_tuning cur;
  read_tuning(m, &cur);
  pbfb_tuning best = cur;
  Surface* sm = &m->sm;
  Surface* ss = &m->ss;
  // both surfaces, single and double layer at once (as in the coupled operator)
  auto far = [&](int precision) {
    return [&, precision]() -> int {
      PB_TRY(launch_bem_far(m, sm, x.p, x.p + sm->col0, -1.0, 1.0, 0.0, precision, y.p + sm->col0, false));
      return launch_bem_far(m, ss, x.p, x.p + ss->col0, 1.0, -1.0, m->kappa, precision, y.p + ss->col0, false);
    };
  };
  double t_best[3] = {1e300, 1e300, 1e300};
  // float32 far field
  for (int tpt : {1, 2, 4})
    for (int packed : {0, 1, 2}) {
      if (packed == 1 && tpt < 2) continue;
      if (packed == 2 && tpt != 4) continue;
      // split kernels: 0 = whole waves of resident blocks
      static const int bps_split[4] = {0, 8, 16, 32}, bps_mutual[4] = {16, 32, 64, 64};
      for (int bi = 0; bi < (packed == 2 ? 3 : 4); ++bi) {
        const int bps = packed == 2 ? bps_mutual[bi] : bps_split[bi];
        pbfb_tuning t = best;
        t.nbody_targets_per_thread = tpt;
        t.nbody_packed = packed;
        t.nbody_blocks_per_sm = bps;
        t.treecode = 1;
        write_tuning(m, &t);
        double ms;
        int st = time_ms(m, reps, far(PBFB_MIXED), &ms);
        if (st) {
          write_tuning(m, &cur);
          return st;
        }
        if (ms < t_best[0]) {
          t_best[0] = ms;
          best.nbody_targets_per_thread = tpt;
          best.nbody_packed = packed;
          best.nbody_blocks_per_sm = bps;
          best.treecode = 1;
        }
      }
    }
  // the treecode with two or four targets per thread (surfaces too small for a tree leaf keep the
  // direct sum), against the best direct shape; its plan is built on the first (untimed) run
  for (int tc : {2, 3}) {
    pbfb_tuning t = best;
    t.treecode = tc;
    write_tuning(m, &t);
    double ms;
    int st = time_ms(m, reps, far(PBFB_MIXED), &ms);
    if (st) {
      write_tuning(m, &cur);
      return st;
    }
    if (ms < t_best[0]) {
      t_best[0] = ms;
      best.treecode = tc;
    }
  }
  // float-float far field
  for (int kind : {1, 2, 3, 4})
    for (int bps : {4, 8, 16, 24}) {
      pbfb_tuning t = best;
      t.ff_kernel = kind;
      t.ff_blocks_per_sm = bps;
      write_tuning(m, &t);
      double ms;
      int st = time_ms(m, reps, far(PBFB_FLOAT2), &ms);
      if (st) {
        write_tuning(m, &cur);
        return st;
      }
      if (ms < t_best[1]) {
        t_best[1] = ms;
        best.ff_kernel = kind;
        best.ff_blocks_per_sm = bps;
      }
    }
  // SpMV of the operator's sparse part (10 products per repetition)
  for (int L : {4, 8, 16})
    for (int B : {128, 256, 512}) {
      pbfb_tuning t = best;
      t.spmv_lanes = L;
      t.spmv_block = B;
      write_tuning(m, &t);
      double ms;
      int st = time_ms(m, reps, [&]() -> int {
        for (int k = 0; k < 10; ++k) PB_TRY(launch_spmv(m, x.p, y.p));
        return PBFB_OK;
      }, &ms);
      if (st) {
        write_tuning(m, &cur);
        return st;
      }
      if (ms < t_best[2]) {
        t_best[2] = ms;
        best.spmv_lanes = L;
        best.spmv_block = B;
      }
    }
  // cooperative inner PCG of the block preconditioner (20 iterations); skipped on meshes solved
  // without the grid-barrier kernel
  double t_pcg = 0.0;
  if (!m->no_coop) {
    t_pcg = 1e300;
    for (int lanes : {8, 4, 2, 1})
    for (int bps : {1, 2, 4, 8, 0}) {
      pbfb_tuning t = best;
      t.pcg_blocks_per_sm = bps;
      t.pcg_lanes = lanes;
      write_tuning(m, &t);
      double ms;
      int st = time_ms(m, reps, [&]() -> int { return block_precond_apply(m, x.p, y.p, 20, true); }, &ms);
      if (st) {
        write_tuning(m, &cur);
        return st;
      }
      if (ms < t_pcg) {
        t_pcg = ms;
        best.pcg_blocks_per_sm = bps;
        best.pcg_lanes = lanes;
      }
    }
  }
  write_tuning(m, &best);
  if (best_out) *best_out = best;
  if (ms_out) {
    ms_out[0] = t_best[0];
    ms_out[1] = t_best[1];
    ms_out[2] = t_best[2] / 10.0;
    ms_out[3] = t_pcg;
  }
  return PBFB_OK;
}

}  // namespace pbfb

extern "C" {

int pbfb_get_tuning(const pbfb_mesh* h, pbfb_tuning* out) {
  pbfb::Mesh* m = pbfb_mesh_internal(const_cast<pbfb_mesh*>(h));
  if (!m || !out) {
    pbfb::set_error("get_tuning: bad argument");
    return PBFB_ERR_INVALID;
  }
  pbfb::read_tuning(m, out);
  return PBFB_OK;
}

int pbfb_apply_tuning(pbfb_mesh* h, const pbfb_tuning* t) {
  pbfb::Mesh* m = pbfb_mesh_internal(h);
  if (!m || !t || !pbfb::valid_tuning(t)) {
    pbfb::set_error("apply_tuning: bad argument or a field out of range");
    return PBFB_ERR_INVALID;
  }
  pbfb::write_tuning(m, t);
  return PBFB_OK;
}

int pbfb_autotune(pbfb_mesh* h, int reps, pbfb_tuning* best, double* ms) {
  pbfb::Mesh* m = pbfb_mesh_internal(h);
  if (!m || reps < 1 || reps > 20) {
    pbfb::set_error("autotune: bad argument");
    return PBFB_ERR_INVALID;
  }
  if (cudaSetDevice(m->dev) != cudaSuccess) {
    pbfb::set_error("autotune: cudaSetDevice failed");
    return PBFB_ERR_CUDA;
  }
  if (!m->params) {
    pbfb::set_error("call pbfb_set_params first");
    return PBFB_ERR_STATE;
  }
  return pbfb::autotune(m, reps, best, ms);
}

}  // extern "C"
