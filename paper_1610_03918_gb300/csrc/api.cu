// C ABI: context set-up (geometry of Sec. III), particle loading, the step
// driver and diagnostics.  Kernels live in particles.cu and poisson.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace picgb {

thread_local std::string g_last_error;

cudaError_t note(cudaError_t e, const char *where) {
  if (e != cudaSuccess) g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e;
}

void *tmp_alloc(pic_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void *p = nullptr;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->stream, c->cfg.alloc_user);
    // the kernels move 16-byte vectors: a block the caller's allocator did
    // not align is given back and counts as a failed allocation
    if (p && (reinterpret_cast<uintptr_t>(p) & 15)) {
      if (c->cfg.free) c->cfg.free(p, c->stream, c->cfg.alloc_user);
      p = nullptr;
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  return p;
}

void tmp_free(pic_ctx *c, void *p) {
  if (!p) return;
  if (c->cfg.alloc) {
    if (c->cfg.free) c->cfg.free(p, c->stream, c->cfg.alloc_user);
  } else {
    cudaFree(p);
  }
}

void *dev_alloc(pic_ctx *c, size_t bytes) {
  void *p = tmp_alloc(c, bytes);
  if (p) c->allocs.push_back(p);
  return p;
}

namespace {

constexpr int64_t kStageParticles = int64_t(1) << 22;
constexpr int kTuneSteps = 48;   // particle steps timed after a sort when tuning the interval
constexpr int kTuneMin = 4;      // shortest interval the tuning may choose

// Node arrays held on the device as double-float (hi, lo) pairs
std::vector<float2> to_pairs(const double *x, size_t n) {
  std::vector<float2> p(n);
  for (size_t k = 0; k < n; ++k) p[k] = pair_split(x[k]);
  return p;
}

void from_pairs(const float2 *d, size_t n, double *out) {
  std::vector<float2> p(n);
  cudaMemcpy(p.data(), d, n * sizeof(float2), cudaMemcpyDeviceToHost);
  for (size_t k = 0; k < n; ++k) out[k] = pair_join(p[k]);
}

// Conductor cells: the electrode slab i >= nx - depth with the trench
// columns [y0, y0 + width) open (Sec. III-C).
bool plasma_cell(const pic_config &cfg, int i, int j) {
  if (i < 0 || i >= cfg.nx || j < 0 || j >= cfg.ny) return false;
  if (cfg.trench_depth > 0 && i >= cfg.nx - cfg.trench_depth) {
    return cfg.trench_width > 0 && j >= cfg.trench_y0 && j < cfg.trench_y0 + cfg.trench_width;
  }
  return true;
}

bool plasma_cell_wrapped(const pic_config &cfg, int i, int j) {
  if (cfg.periodic_x) i = ((i % cfg.nx) + cfg.nx) % cfg.nx;
  if (cfg.periodic_y) j = ((j % cfg.ny) + cfg.ny) % cfg.ny;
  return plasma_cell(cfg, i, j);
}

// Node classification: Dirichlet mask and values, open mesh edges, lift.
// Values where categories meet: conductor-adjacent and x = nx nodes take the
// electrode value, x = 0 nodes the top-plate value, bounded-y walls 0.
void build_geometry(pic_ctx *c, std::vector<uint8_t> &cellmask, std::vector<double> &lift) {
  const pic_config &cfg = c->cfg;
  const Geom &g = c->g;
  cellmask.assign(size_t(g.nx) * g.ny, 0);
  for (int i = 0; i < g.nx; ++i)
    for (int j = 0; j < g.ny; ++j)
      cellmask[size_t(i) * g.ny + j] = plasma_cell(cfg, i, j) ? kCellPlasma : 0;
  // interior cells: every neighbour within one cell is plasma (moves of at
  // most one cell from them cannot reach a wall)
  for (int i = 0; i < g.nx; ++i)
    for (int j = 0; j < g.ny; ++j) {
      bool all = true;
      for (int di = -1; di <= 1 && all; ++di)
        for (int dj = -1; dj <= 1 && all; ++dj) all = plasma_cell_wrapped(cfg, i + di, j + dj);
      if (all) cellmask[size_t(i) * g.ny + j] |= kCellInterior;
    }
  const size_t nn = size_t(g.nxn) * g.nyn;
  std::vector<uint8_t> dir(nn, 0);
  std::vector<double> val(nn, 0.0);
  std::vector<uint8_t> &elec = c->h_electrode;   // held at the electrode potential
  elec.assign(nn, 0);
  for (int i = 0; i < g.nxn; ++i) {
    for (int j = 0; j < g.nyn; ++j) {
      const size_t n = size_t(i) * g.nyn + j;
      if (!g.py && (j == 0 || j == g.nyn - 1)) {
        dir[n] = 1;
        val[n] = 0.0;
      }
      if (!g.px && i == 0) {
        dir[n] = 1;
        val[n] = cfg.phi_top;
      }
      if (!g.px && i == g.nxn - 1) {
        dir[n] = 1;
        val[n] = cfg.phi_electrode;
        elec[n] = 1;
      }
      // touching a conductor cell (in-domain cells only)
      bool touch = false;
      for (int di = -1; di <= 0; ++di)
        for (int dj = -1; dj <= 0; ++dj) {
          int ci = i + di, cj = j + dj;
          if (g.px) ci = (ci + g.nx) % g.nx;
          if (g.py) cj = (cj + g.ny) % g.ny;
          if (ci < 0 || ci >= g.nx || cj < 0 || cj >= g.ny) continue;
          if (!cellmask[size_t(ci) * g.ny + cj]) touch = true;
        }
      if (touch) {
        dir[n] = 1;
        val[n] = cfg.phi_electrode;
        elec[n] = 1;
      }
    }
  }
  c->h_nodeflags.assign(nn, 0);
  c->h_g.assign(nn, 0.0);
  lift.assign(nn, 0.0);
  for (int i = 0; i < g.nxn; ++i) {
    for (int j = 0; j < g.nyn; ++j) {
      const size_t n = size_t(i) * g.nyn + j;
      uint8_t f = dir[n] ? 0 : kFree;
      // x edge (i, j) - (i+1, j) borders cells (i, j-1) and (i, j)
      const bool has_xp = g.px || i + 1 < g.nxn;
      const bool has_xm = g.px || i - 1 >= 0;
      const bool has_yp = g.py || j + 1 < g.nyn;
      const bool has_ym = g.py || j - 1 >= 0;
      if (has_xp && (plasma_cell_wrapped(cfg, i, j - 1) || plasma_cell_wrapped(cfg, i, j)))
        f |= kOpenXp;
      if (has_xm && (plasma_cell_wrapped(cfg, i - 1, j - 1) || plasma_cell_wrapped(cfg, i - 1, j)))
        f |= kOpenXm;
      // y edge (i, j) - (i, j+1) borders cells (i-1, j) and (i, j)
      if (has_yp && (plasma_cell_wrapped(cfg, i - 1, j) || plasma_cell_wrapped(cfg, i, j)))
        f |= kOpenYp;
      if (has_ym && (plasma_cell_wrapped(cfg, i - 1, j - 1) || plasma_cell_wrapped(cfg, i, j - 1)))
        f |= kOpenYm;
      c->h_nodeflags[n] = f;
      c->h_g[n] = dir[n] ? val[n] : 0.0;
    }
  }
  for (int i = 0; i < g.nxn; ++i) {
    for (int j = 0; j < g.nyn; ++j) {
      const size_t n = size_t(i) * g.nyn + j;
      if (dir[n]) continue;
      const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
      double s = 0.0;
      for (auto &q : nb) {
        int a = q[0], b = q[1];
        if (g.px) a = (a + g.nxn) % g.nxn;
        if (g.py) b = (b + g.nyn) % g.nyn;
        const size_t m = size_t(a) * g.nyn + b;
        if (dir[m]) s += val[m];
      }
      lift[n] = s;
    }
  }
}

pic_status check(cudaError_t e) { return e == cudaSuccess ? PIC_OK : PIC_ECUDA; }

pic_status status_from_bits(uint32_t bits) {
  if (bits & PIC_ST_NOCONV) return PIC_ENOCONV;
  if (bits & PIC_ST_CFL) return PIC_ECFL;
  if (bits & PIC_ST_CAPACITY) return PIC_EOVERFLOW;
  if (bits & PIC_ST_RANGE) return PIC_ERANGE;
  if (bits & PIC_ST_FULL) return PIC_EFULL;
  return PIC_OK;
}

pic_status validate(const pic_config *cfg) {
  if (!cfg) return PIC_EINVAL;
  if (cfg->nx < 2 || cfg->ny < 2) return PIC_EINVAL;
  // particle cells are packed as (i << 16) | j
  if (cfg->nx > 32767 || cfg->ny > 65535) return PIC_EINVAL;
  if (int64_t(cfg->nx + 1) * int64_t(cfg->ny + 1) >= (int64_t(1) << 30)) return PIC_EINVAL;
  // red-black colouring of a periodic direction needs an even node count
  if (cfg->periodic_x && (cfg->nx % 2)) return PIC_EINVAL;
  if (cfg->periodic_y && (cfg->ny % 2)) return PIC_EINVAL;
  if (!(cfg->dt > 0) || !(cfg->poisson_rtol > 0)) return PIC_EINVAL;
  if (cfg->poisson_maxit < 1 || cfg->sort_every < 0) return PIC_EINVAL;
  if (cfg->warm_start < 0 || cfg->warm_start > 4) return PIC_EINVAL;
  if (cfg->warm_start == 3 && !cfg->unet_weights) return PIC_EINVAL;
  if (cfg->decomposed && cfg->sort_every < 1) return PIC_EINVAL;
  if (cfg->tile_variant < 0 || cfg->tile_variant >= kNumTileVariants) return PIC_EINVAL;
  if (!std::isfinite(cfg->phi_rf_amp) || !std::isfinite(cfg->omega_rf)) return PIC_EINVAL;
  if (cfg->recycle) {
    const int plasma_rows = cfg->nx - cfg->trench_depth;
    const int x1 = cfg->source_x1 ? cfg->source_x1 : plasma_rows;
    if (cfg->source_x0 < 0 || x1 <= cfg->source_x0 || x1 > plasma_rows) return PIC_EINVAL;
    if (!(cfg->recycle_vth >= 0) || !std::isfinite(cfg->recycle_vth)) return PIC_EINVAL;
  }
  if (cfg->poisson_method < 0 || cfg->poisson_method > 1) return PIC_EINVAL;
  for (int s = 0; s < 2; ++s) {
    if (cfg->ppc[s] < 1 || cfg->capacity[s] < 0) return PIC_EINVAL;
    if (cfg->capacity[s] > (int64_t(1) << 31) - (int64_t(1) << 26)) return PIC_EINVAL;
    if (!(cfg->charge[s] == cfg->charge[s]) || !(cfg->alpha[s] == cfg->alpha[s])) return PIC_EINVAL;
  }
  if (cfg->trench_depth < 0 || cfg->trench_depth > cfg->nx) return PIC_EINVAL;
  if (cfg->trench_width < 0 || cfg->trench_y0 < 0 || cfg->trench_y0 + cfg->trench_width > cfg->ny)
    return PIC_EINVAL;
  if (cfg->trench_depth > 0 && cfg->periodic_x) return PIC_EINVAL;
  if (cfg->hit_capacity < 0) return PIC_EINVAL;
  if (cfg->alloc && !cfg->free) return PIC_EINVAL;
  return PIC_OK;
}

pic_status prepare(pic_ctx *c) {
  if (!c->fields_dirty) return PIC_OK;
  pic_status st;
  if ((st = check(launch_sort(c))) != PIC_OK) return st;
  c->steps_since_sort = 0;
  c->needs_sort = 0;
  if ((st = check(launch_particles(c, 1, 0.f, nullptr))) != PIC_OK) return st;
  if ((st = check(launch_rf_bias(c, 0))) != PIC_OK) return st;
  if ((st = check(launch_rho(c, 0))) != PIC_OK) return st;
  st = poisson_solve(c, true);
  if (st != PIC_OK) return st;
  // the extrapolated warm start begins from a constant history
  if (cudaMemcpyAsync(c->d_phi_prev, c->d_phi, size_t(c->g.nxn) * c->g.nyn * sizeof(float2),
                      cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return PIC_ECUDA;
  if (c->pending_kick[0] || c->pending_kick[1]) {
    if ((st = check(launch_particles(c, 2, -0.5f, c->pending_kick))) != PIC_OK) return st;
    c->pending_kick[0] = c->pending_kick[1] = 0;
  }
  c->fields_dirty = 0;
  return PIC_OK;
}

// Ends the capture on stream s and returns its current leaf nodes in `leaves`.
cudaError_t capture_leaves(cudaStream_t s, std::vector<cudaGraphNode_t> &leaves) {
  cudaStreamCaptureStatus cs;
  unsigned long long id;
  cudaGraph_t gg;
  const cudaGraphNode_t *d = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, &id, &gg, &d, &ed, &nd);
  if (e == cudaSuccess) leaves.assign(d, d + nd);
  cudaGraph_t out;
  const cudaError_t e2 = cudaStreamEndCapture(s, &out);
  return e == cudaSuccess ? e2 : e;
}

// One step from the host: sort (when due), particle kernel, rho, solve (which
// leaves the field), with the phase events ev (kPhaseEvents of them).
pic_status step_kernels(pic_ctx *c, bool sorting, cudaEvent_t *ev) {
  pic_status st;
  cudaEventRecord(ev[0], c->stream);
  if (sorting) {
    if ((st = check(launch_sort(c))) != PIC_OK) return st;
    c->launches += 4;
  }
  cudaEventRecord(ev[1], c->stream);
  if ((st = check(launch_particles(c, 0, 1.f, nullptr))) != PIC_OK) return st;
  cudaEventRecord(ev[2], c->stream);
  if ((st = check(launch_rf_bias(c, 1))) != PIC_OK) return st;
  if ((st = check(launch_rho(c, 1))) != PIC_OK) return st;
  cudaEventRecord(ev[3], c->stream);
  st = poisson_solve(c, c->cfg.warm_start == 0);
  if (st != PIC_OK) return st;
  cudaEventRecord(ev[4], c->stream);
  c->launches += 2;
  return PIC_OK;
}

// Appends one step of context c to graph g after the nodes in `deps`:
// [sort] -> particle kernel -> rho -> the Poisson solve as nested conditional
// nodes (its residual passes write the field; with the direct solve and the
// previous potential as the guess its first pass forms rho).  With `events`, external event
// nodes recording c->tev separate the phases (PIC_DIAG_TIMING); the launch
// points them at a slot of the event pool.  On return `deps` holds the step's last node(s).
// Kernel arguments are fixed device pointers; the particle buffers are reached
// through the device-side buffer table, so the sort's swap needs no re-capture.
// part 0: the whole step; 1: its particle phase (a decomposed run's, which
// ends by copying the rank's bottom counts into the exchange buffer); 2: its
// field phase.
cudaError_t capture_step(pic_ctx *c, cudaGraph_t g, std::vector<cudaGraphNode_t> &deps,
                         int with_sort, bool events, int part = 0) {
  const int cur_save[2] = {c->cur[0], c->cur[1]};
  const int64_t launches_save = c->launches;
  auto rec = [&](int k) {
    if (events) cudaEventRecordWithFlags(c->tev[k], c->stream, cudaEventRecordExternal);
  };
  cudaError_t e = cudaStreamBeginCaptureToGraph(c->stream, g, deps.empty() ? nullptr : deps.data(),
                                                nullptr, deps.size(), cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rec(0);
    if (part != 2) {
      if (with_sort) launch_sort(c);
      rec(1);
      launch_particles(c, 0, 1.f, nullptr);
      rec(2);
    }
    if (part == 1) {
      const size_t nn = size_t(c->g.nxn) * c->g.nyn;
      cudaMemcpyAsync(c->d_acc + 2 * nn, c->d_bottom, 2 * size_t(c->g.ny) * 8, cudaMemcpyDeviceToDevice,
                      c->stream);
    } else {
      launch_rf_bias(c, 1);
      if (!rho_in_solve(c)) launch_rho(c, 1, c->cfg.warm_start == 1);   // opens the solve captured next
    }
    rec(3);
    e = note(capture_leaves(c->stream, deps), "capture: particle phase");
  }
  if (e == cudaSuccess && part != 1) e = note(poisson_capture(c, g, deps), "capture: Poisson conditionals");
  if (e == cudaSuccess && events) {
    e = cudaStreamBeginCaptureToGraph(c->stream, g, deps.data(), nullptr, deps.size(),
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rec(4);
      e = capture_leaves(c->stream, deps);
    }
  }
  c->cur[0] = cur_save[0];
  c->cur[1] = cur_save[1];
  c->launches = launches_save;
  cudaGetLastError();
  return e;
}

// Capture (once) and instantiate the step graph of one context, with or
// without the phase event nodes; the event nodes are looked up by the
// placeholder event each records.
cudaError_t step_graph(pic_ctx *c, int with_sort, int events) {
  if (c->gexec[with_sort][events]) return cudaSuccess;
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> deps;
  e = note(capture_step(c, g, deps, with_sort, events != 0), "step graph capture");
  if (e == cudaSuccess && events) {
    size_t n = 0;
    e = cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess) e = cudaGraphGetNodes(g, nodes.data(), &n);
    int found = 0;
    for (size_t k = 0; e == cudaSuccess && k < n; ++k) {
      cudaGraphNodeType t;
      cudaEvent_t ev;
      if (cudaGraphNodeGetType(nodes[k], &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
      if (cudaGraphEventRecordNodeGetEvent(nodes[k], &ev) != cudaSuccess) continue;
      for (int q = 0; q < kPhaseEvents; ++q)
        if (ev == c->tev[q]) {
          c->evnode[with_sort][q] = nodes[k];
          found |= 1 << q;
        }
    }
    if (e == cudaSuccess && found != (1 << kPhaseEvents) - 1) e = cudaErrorInvalidValue;
    note(e, "step graph event nodes");
  }
  if (e == cudaSuccess)
    e = note(cudaGraphInstantiate(&c->gexec[with_sort][events], g, 0), "step graph instantiate");
  if (e == cudaSuccess) c->graph[with_sort][events] = g;
  else cudaGraphDestroy(g);
  cudaGetLastError();
  return e;
}

// Reads the phase times of the recorded timing slots (waiting for the last)
// into the PIC_DIAG_TIMING totals and feeds the sort-interval tuning.
pic_status flush_timing(pic_ctx *c) {
  if (c->tpend == 0) return PIC_OK;
  if (cudaEventSynchronize(c->tpool[c->tpend - 1][kPhaseEvents - 1]) != cudaSuccess) return PIC_ECUDA;
  for (int s = 0; s < c->tpend; ++s) {
    float ms[kPhaseEvents - 1] = {};
    for (int q = 0; q + 1 < kPhaseEvents; ++q) cudaEventElapsedTime(&ms[q], c->tpool[s][q], c->tpool[s][q + 1]);
    c->t_sort += ms[0];
    c->t_part += ms[1];
    c->t_other += ms[2];
    if (c->cfg.graphs) {
      c->t_poisson += ms[3];
      c->last_ms = ms[3];
    } else {
      c->t_poisson += c->last_ms;   // the solve's own time, without the host polling
    }
    if (c->tslot_tune[s] && c->tune_state < 2) {
      // a sort opens the measurement, then the particle times of the steps after it
      if (c->tune_state == 0) {
        c->tune_state = 1;
        c->tune_sort_ms = ms[0];
        c->tune_particle_ms.clear();
      }
      c->tune_particle_ms.push_back(ms[1]);
      if (int(c->tune_particle_ms.size()) >= kTuneSteps) {
        double sum = 0.0, best = 0.0;
        int best_s = kTuneMin;
        for (int k = 1; k <= kTuneSteps; ++k) {
          sum += c->tune_particle_ms[k - 1];
          const double per_step = (c->tune_sort_ms + sum) / k;
          if (k >= kTuneMin && (k == kTuneMin || per_step < best)) {
            best = per_step;
            best_s = k;
          }
        }
        c->sort_interval = best_s;
        c->tune_state = 2;
      }
    }
  }
  c->tpend = 0;
  return PIC_OK;
}

// Adds the kernels of the solves that graph steps ran since the last count
// (from the solver's running totals on the device) to the launch count.
pic_status count_solves(pic_ctx *c) {
  PoissonState ps;
  if (cudaMemcpy(&ps, c->d_ps, sizeof(ps), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  c->launches += poisson_kernel_count(c, ps.n_solves - c->seen_solves, ps.sum_outer - c->seen_outer,
                                      ps.sum_total - c->seen_total);
  c->seen_solves = ps.n_solves;
  c->seen_outer = ps.sum_outer;
  c->seen_total = ps.sum_total;
  c->last_outer = ps.outer_iters;
  return PIC_OK;
}

}  // namespace
}  // namespace picgb

using namespace picgb;

struct pic_batch {
  std::vector<pic_ctx *> m;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int dev = 0;
  int sort_every = 1;
  int steps_since_sort = 0;
  int timing = 0;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double t_ms = 0.0;
  int64_t t_steps = 0;
};

namespace picgb {
namespace {

// The ensemble graph: an event node, then every member's step as an
// independent branch, then an event node after all of them.
cudaError_t batch_graph(pic_batch *b, int with_sort) {
  if (b->gexec[with_sort]) return cudaSuccess;
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> root, leaves;
  e = cudaStreamBeginCaptureToGraph(b->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecordWithFlags(b->ev[0], b->stream, cudaEventRecordExternal);
    e = capture_leaves(b->stream, root);
  }
  for (size_t k = 0; e == cudaSuccess && k < b->m.size(); ++k) {
    std::vector<cudaGraphNode_t> d = root;
    e = capture_step(b->m[k], g, d, with_sort, false);
    leaves.insert(leaves.end(), d.begin(), d.end());
  }
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(b->stream, g, leaves.data(), nullptr, leaves.size(),
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaEventRecordWithFlags(b->ev[1], b->stream, cudaEventRecordExternal);
      std::vector<cudaGraphNode_t> tail;
      e = capture_leaves(b->stream, tail);
    }
  }
  note(e, "ensemble graph capture");
  if (e == cudaSuccess) e = note(cudaGraphInstantiate(&b->gexec[with_sort], g, 0), "ensemble graph instantiate");
  if (e == cudaSuccess) b->graph[with_sort] = g;
  else cudaGraphDestroy(g);
  cudaGetLastError();
  return e;
}

}  // namespace
}  // namespace picgb

extern "C" {

pic_status pic_batch_init(const pic_config *cfgs, int32_t n, void *stream, pic_batch **out) {
  if (!out || !cfgs || n < 1) return PIC_EINVAL;
  *out = nullptr;
  for (int32_t k = 0; k < n; ++k) {
    if (cfgs[k].sort_every < 1 || cfgs[k].sort_every != cfgs[0].sort_every ||
        cfgs[k].device != cfgs[0].device || cfgs[k].decomposed)
      return PIC_EINVAL;
    const pic_status st = validate(&cfgs[k]);
    if (st != PIC_OK) return st;
  }
  pic_batch *b = new (std::nothrow) pic_batch();
  if (!b) return PIC_ENOMEM;
  b->dev = cfgs[0].device;
  b->sort_every = cfgs[0].sort_every;
  b->timing = cfgs[0].timing;
  if (cudaSetDevice(b->dev) != cudaSuccess) {
    delete b;
    return PIC_ECUDA;
  }
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  cudaEventCreate(&b->ev[0]);
  cudaEventCreate(&b->ev[1]);
  for (int32_t k = 0; k < n; ++k) {
    pic_config cfg = cfgs[k];
    cfg.stream = b->stream;
    cfg.graphs = 1;
    cfg.timing = 0;
    pic_ctx *c = nullptr;
    const pic_status st = pic_init(&cfg, &c);
    if (st != PIC_OK) {
      pic_batch_free(b);
      return st;
    }
    b->m.push_back(c);
  }
  *out = b;
  return PIC_OK;
}

pic_ctx *pic_batch_member(pic_batch *b, int32_t k) {
  if (!b || k < 0 || k >= int32_t(b->m.size())) return nullptr;
  return b->m[k];
}

pic_status pic_batch_step(pic_batch *b, int32_t nsteps) {
  if (!b || nsteps < 0) return PIC_EINVAL;
  if (cudaSetDevice(b->dev) != cudaSuccess) return PIC_ECUDA;
  bool prepared = false;
  for (pic_ctx *c : b->m) {
    if (!c->fields_dirty) continue;
    const pic_status st = prepare(c);
    if (st != PIC_OK) return st;
    prepared = true;
  }
  if (prepared) {
    b->steps_since_sort = 0;
    for (pic_ctx *c : b->m) c->steps_since_sort = 0;
  }
  for (int32_t k = 0; k < nsteps; ++k) {
    int sorting = b->steps_since_sort >= b->sort_every ? 1 : 0;
    for (pic_ctx *c : b->m) {   // a member restored from a checkpoint
      if (c->needs_sort) sorting = 1;
      c->needs_sort = 0;
    }
    if (check(batch_graph(b, sorting)) != PIC_OK) return PIC_ECUDA;
    if (note(cudaGraphLaunch(b->gexec[sorting], b->stream), "ensemble graph launch") != cudaSuccess)
      return PIC_ECUDA;
    for (pic_ctx *c : b->m) {
      if (sorting) {
        c->cur[0] ^= 1;
        c->cur[1] ^= 1;
        c->steps_since_sort = 0;
      }
      c->steps_since_sort += 1;
      c->step += 1;
    }
    b->steps_since_sort = sorting ? 1 : b->steps_since_sort + 1;
    if (b->timing) {
      if (note(cudaEventSynchronize(b->ev[1]), "ensemble step") != cudaSuccess) return PIC_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
      b->t_ms += ms;
      b->t_steps += 1;
    }
  }
  return PIC_OK;
}

pic_status pic_batch_timing(pic_batch *b, double *out) {
  if (!b || !out) return PIC_EINVAL;
  if (cudaSetDevice(b->dev) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess)
    return PIC_ECUDA;
  out[0] = double(b->t_steps);
  out[1] = b->t_ms;
  b->t_steps = 0;
  b->t_ms = 0.0;
  return PIC_OK;
}

pic_status pic_batch_free(pic_batch *b) {
  if (!b) return PIC_OK;
  cudaSetDevice(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k) {
    if (b->gexec[k]) cudaGraphExecDestroy(b->gexec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
  }
  for (pic_ctx *c : b->m) pic_free(c);
  for (int k = 0; k < 2; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return PIC_OK;
}


const char *pic_last_error(void) { return g_last_error.c_str(); }

pic_status pic_learned_input(pic_ctx *c, int32_t hpad, float *x, double *scale) {
  if (!c || !x || !scale) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  return learned_input(c, hpad, x, scale);
}

pic_status pic_poisson(pic_ctx *c, int32_t guess, const float *y, double scale, double *stats) {
  if (!c || guess < 0 || guess > 3) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  if (c->fields_dirty) {
    const pic_status st = pic_step(c, 0);
    if (st != PIC_OK) return st;
  }
  return poisson_with_guess(c, guess, y, scale, stats);
}

const char *pic_strerror(pic_status st) {
  switch (st) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "device allocation failed";
    case PIC_ECUDA: return "CUDA error";
    case PIC_ENOCONV: return "Poisson solve did not reach the tolerance";
    case PIC_EOVERFLOW: return "particle capacity exceeded";
    case PIC_ECFL: return "a particle moved farther than the face-walk limit";
    case PIC_ETIMEOUT: return "bounded device wait gave up";
    case PIC_EFULL: return "hit-record buffer full";
    case PIC_ESTATE: return "call not valid in the current state";
    case PIC_ERANGE: return "particle outside the plasma region";
    case PIC_ESIZE: return "grid has more nodes than the fixed deposit scratch (2^20)";
  }
  return "unknown status";
}

pic_status pic_init(const pic_config *cfg, pic_ctx **out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  pic_status st = validate(cfg);
  if (st != PIC_OK) return st;
  pic_ctx *c = new (std::nothrow) pic_ctx();
  if (!c) return PIC_ENOMEM;
  c->cfg = *cfg;
  c->dev = cfg->device;
  if (cudaSetDevice(c->dev) != cudaSuccess) {
    delete c;
    return PIC_ECUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
    c->own_stream = false;
  } else {
    cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    c->own_stream = true;
  }
  Geom &g = c->g;
  g.nx = cfg->nx;
  g.ny = cfg->ny;
  g.px = cfg->periodic_x ? 1 : 0;
  g.py = cfg->periodic_y ? 1 : 0;
  g.nxn = g.px ? g.nx : g.nx + 1;
  g.nyn = g.py ? g.ny : g.ny + 1;
  g.dnyn = make_fastdiv(uint32_t(g.nyn));
  // tile arrays sized for the smallest tile shape; the variant in use sets ntx, nty
  const int ntiles = ((g.nx + (1 << kMinTileLog2) - 1) >> kMinTileLog2) *
                     ((g.ny + (1 << kMinTileLog2) - 1) >> kMinTileLog2);
  c->max_tiles = ntiles;
  set_tile_variant(c, cfg->tile_variant);
  const size_t nn = size_t(g.nxn) * g.nyn;

  std::vector<uint8_t> cellmask;
  std::vector<double> lift;
  build_geometry(c, cellmask, lift);

  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = dev_alloc(c, bytes);
    if (!p) ok = false;
    return p;
  };
  c->d_cellmask = (uint8_t *)A(cellmask.size());
  c->d_nodeflags = (uint8_t *)A(nn);
  c->d_lift = (float *)A(nn * 4);
  c->d_g = (float2 *)A(nn * 8);
  c->d_acc = (unsigned long long *)A((2 * nn + 2 * size_t(g.ny)) * 8);
  c->d_rho_ext = (float2 *)A(nn * 8);
  c->d_rho = (float2 *)A(nn * 8);
  c->d_phi = (float2 *)A(nn * 8);
  c->d_E = (float2 *)A(nn * sizeof(float2));
  c->d_fe = (double *)A(2 * 8);
  for (int s = 0; s < 2; ++s) {
    c->cap[s] = ((cfg->capacity[s] + 4 * int64_t(ntiles) + 3) / 4) * 4;
    for (int b = 0; b < 2; ++b) {
      ParticleBuf &P = c->pb[s][b];
      P.cell = (int32_t *)A(c->cap[s] * 4);
      P.fx = (float *)A(c->cap[s] * 4);
      P.fy = (float *)A(c->cap[s] * 4);
      P.vx = (float *)A(c->cap[s] * 4);
      P.vy = (float *)A(c->cap[s] * 4);
      P.id = (uint32_t *)A(c->cap[s] * 4);
    }
    c->cur[s] = 0;
  }
  c->d_pbufs = (ParticleBuf *)A(4 * sizeof(ParticleBuf));
  c->d_cur = (int32_t *)A(2 * sizeof(int32_t));
  c->d_tile_count = (uint32_t *)A(2 * size_t(ntiles) * 4);
  c->d_tile_cursor = (uint32_t *)A(2 * size_t(ntiles) * 4);
  c->d_tile_start = (uint32_t *)A(2 * size_t(ntiles) * 4);
  c->max_chunks = 0;
  for (int s = 0; s < 2; ++s) c->max_chunks += ntiles + c->cap[s] / kChunk + 1;
  c->d_chunks = (Chunk *)A(size_t(c->max_chunks) * sizeof(Chunk));
  c->d_nchunks = (int32_t *)A(4);
  c->d_nslots = (int64_t *)A(4 * 8);
  c->d_ke_part = (double *)A(size_t(c->max_chunks) * 8);
  c->d_step = (int32_t *)A(4);
  c->d_walls = (unsigned long long *)A(2 * PIC_NWALLS * 8);
  c->d_bottom = (unsigned long long *)A(2 * size_t(g.ny) * 8);
  c->d_hits = (pic_hit *)A(std::max<int64_t>(cfg->hit_capacity, 1) * sizeof(pic_hit));
  c->d_nhits = (unsigned long long *)A(8);
  c->d_status = (uint32_t *)A(4);
  c->src_x0 = cfg->source_x0;
  c->src_x1 = cfg->source_x1 ? cfg->source_x1 : cfg->nx - cfg->trench_depth;
  // RF bias: the electrode's Dirichlet nodes, and the free nodes next to them
  // with their number of electrode neighbours (the lift changes by that
  // count times the RF part)
  std::vector<int32_t> rf_dir, rf_lift;
  std::vector<float2> rf_g0;
  std::vector<float> rf_cnt, rf_lift0;
  if (cfg->phi_rf_amp != 0.0) {
    for (int i = 0; i < g.nxn; ++i)
      for (int j = 0; j < g.nyn; ++j) {
        const size_t n = size_t(i) * g.nyn + j;
        if (!(c->h_nodeflags[n] & kFree)) {
          if (c->h_electrode[n]) {
            rf_dir.push_back(int32_t(n));
            rf_g0.push_back(pair_split(c->h_g[n]));
          }
          continue;
        }
        const int nb[4][2] = {{i - 1, j}, {i + 1, j}, {i, j - 1}, {i, j + 1}};
        int cnt = 0;
        for (auto &q : nb) {
          int a = q[0], b = q[1];
          if (g.px) a = (a + g.nxn) % g.nxn;
          if (g.py) b = (b + g.nyn) % g.nyn;
          if (a < 0 || a >= g.nxn || b < 0 || b >= g.nyn) continue;
          const size_t m = size_t(a) * g.nyn + b;
          if (!(c->h_nodeflags[m] & kFree) && c->h_electrode[m]) ++cnt;
        }
        if (cnt) {
          rf_lift.push_back(int32_t(n));
          rf_cnt.push_back(float(cnt));
          rf_lift0.push_back(float(lift[n]));
        }
      }
  }
  c->n_rf_dir = int(rf_dir.size());
  c->n_rf_lift = int(rf_lift.size());
  if (c->n_rf_dir) {
    c->d_rf_dir = (int32_t *)A(rf_dir.size() * 4);
    c->d_rf_g0 = (float2 *)A(rf_g0.size() * 8);
  }
  if (c->n_rf_lift) {
    c->d_rf_lift = (int32_t *)A(rf_lift.size() * 4);
    c->d_rf_cnt = (float *)A(rf_cnt.size() * 4);
    c->d_rf_lift0 = (float *)A(rf_lift0.size() * 4);
  }
  c->stage_n = std::min<int64_t>(kStageParticles,
                                 std::max<int64_t>(std::max(cfg->capacity[0], cfg->capacity[1]), 1));
  c->d_stage = (double *)A(size_t(c->stage_n) * 5 * 8);
  c->d_diag = (double *)A(size_t(c->num_sms) * 2 * 2 * 3 * 8);
  if (!ok) {
    pic_free(c);
    return PIC_ENOMEM;
  }
  cudaError_t e = cudaMallocHost((void **)&c->h_status, 4);
  if (e != cudaSuccess) {
    pic_free(c);
    return PIC_ENOMEM;
  }
  cudaMemcpyAsync(c->d_cellmask, cellmask.data(), cellmask.size(), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(c->d_nodeflags, c->h_nodeflags.data(), nn, cudaMemcpyHostToDevice, c->stream);
  {
    std::vector<float> liftf(lift.begin(), lift.end());
    const std::vector<float2> gp = to_pairs(c->h_g.data(), nn);
    cudaMemcpyAsync(c->d_lift, liftf.data(), nn * 4, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_g, gp.data(), nn * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_phi, gp.data(), nn * 8, cudaMemcpyHostToDevice, c->stream);
    if (c->n_rf_dir) {
      cudaMemcpyAsync(c->d_rf_dir, rf_dir.data(), rf_dir.size() * 4, cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(c->d_rf_g0, rf_g0.data(), rf_g0.size() * 8, cudaMemcpyHostToDevice, c->stream);
    }
    if (c->n_rf_lift) {
      cudaMemcpyAsync(c->d_rf_lift, rf_lift.data(), rf_lift.size() * 4, cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(c->d_rf_cnt, rf_cnt.data(), rf_cnt.size() * 4, cudaMemcpyHostToDevice, c->stream);
      cudaMemcpyAsync(c->d_rf_lift0, rf_lift0.data(), rf_lift0.size() * 4, cudaMemcpyHostToDevice, c->stream);
    }
    cudaStreamSynchronize(c->stream);   // the host vectors go out of scope
  }
  cudaMemsetAsync(c->d_acc, 0, (2 * nn + 2 * size_t(g.ny)) * 8, c->stream);
  cudaMemsetAsync(c->d_rho_ext, 0, nn * 8, c->stream);
  cudaMemsetAsync(c->d_rho, 0, nn * 8, c->stream);
  cudaMemsetAsync(c->d_E, 0, nn * sizeof(float2), c->stream);
  cudaMemsetAsync(c->d_fe, 0, 16, c->stream);
  cudaMemsetAsync(c->d_tile_count, 0, 2 * size_t(ntiles) * 4, c->stream);
  cudaMemsetAsync(c->d_tile_cursor, 0, 2 * size_t(ntiles) * 4, c->stream);
  cudaMemsetAsync(c->d_nchunks, 0, 4, c->stream);
  cudaMemsetAsync(c->d_nslots, 0, 32, c->stream);
  cudaMemsetAsync(c->d_step, 0, 4, c->stream);
  cudaMemsetAsync(c->d_walls, 0, 2 * PIC_NWALLS * 8, c->stream);
  cudaMemsetAsync(c->d_bottom, 0, 2 * size_t(g.ny) * 8, c->stream);
  cudaMemsetAsync(c->d_nhits, 0, 8, c->stream);
  cudaMemsetAsync(c->d_status, 0, 4, c->stream);
  for (int s = 0; s < 2; ++s)
    for (int b = 0; b < 2; ++b) cudaMemsetAsync(c->pb[s][b].cell, 0xff, c->cap[s] * 4, c->stream);
  {
    ParticleBuf tab[4] = {c->pb[0][0], c->pb[0][1], c->pb[1][0], c->pb[1][1]};
    int32_t cur0[2] = {0, 0};
    cudaMemcpy(c->d_pbufs, tab, sizeof(tab), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_cur, cur0, sizeof(cur0), cudaMemcpyHostToDevice);
  }
  for (int k = 0; k < kPhaseEvents; ++k) cudaEventCreate(&c->tev[k]);
  e = poisson_setup(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    pic_free(c);
    // an invalid value here means the coarsest multigrid level does not fit
    // in one CTA's shared memory (a grid that cannot be coarsened enough)
    if (e == cudaErrorInvalidValue) return PIC_EINVAL;
    return e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA;
  }
  c->fields_dirty = 1;
  c->needs_sort = 1;
  c->step = 0;
  if (cfg->warm_start == 4) {   // the lift start: its potential is solved now
    c->cfg.warm_start = 1;
    st = pic_set_warm_start(c, 4);
    if (st != PIC_OK) {
      pic_free(c);
      return st;
    }
  }
  if (cfg->warm_start == 3) {
    // the learned guess from a parameter file: a network of this grid's shape
    c->cfg.warm_start = 1;
    c->cfg.unet_weights = nullptr;   // the caller's string is not kept
    pic_unet *net = nullptr;
    st = pic_unet_create(1, (g.nxn + 7) / 8 * 8, g.nyn, c->stream, &net);
    if (st == PIC_OK) st = pic_unet_load(net, cfg->unet_weights);
    if (st == PIC_OK) st = pic_set_learned_start(c, net);
    pic_unet_free(net);
    if (st != PIC_OK) {
      pic_free(c);
      return st;
    }
  }
  *out = c;
  return PIC_OK;
}

pic_status pic_set_learned_start(pic_ctx *c, const pic_unet *net) {
  if (!c || !net) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  const int hpad = (c->g.nxn + 7) / 8 * 8;
  if (unet_batch(net) != 1 || unet_height(net) < hpad || unet_width(net) != c->g.nyn) return PIC_EINVAL;
  pic_status st = PIC_OK;
  if (!c->net) {
    st = pic_unet_create(1, unet_height(net), c->g.nyn, c->stream, &c->net);
    if (st != PIC_OK) return st;
    c->d_net_x = (float *)dev_alloc(c, size_t(unet_height(net)) * c->g.nyn * 2 * 4);
    if (!c->d_net_x) return PIC_ENOMEM;
  }
  if (unet_height(c->net) != unet_height(net)) return PIC_EINVAL;
  if ((st = unet_copy_params(c->net, net)) != PIC_OK) return st;
  if ((st = ensure_vacuum_potential(c)) != PIC_OK) return st;
  // the step graphs hold the old initial guess: capture them again
  if (c->cfg.warm_start == 3) c->cfg.warm_start = 1;
  return pic_set_warm_start(c, 3);
}

pic_status pic_set_warm_start(pic_ctx *c, int32_t mode) {
  if (!c || mode < 0 || mode > 4 || (mode == 3 && !c->net)) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PIC_ECUDA;
  if (mode == c->cfg.warm_start) return PIC_OK;
  if (mode == 4) {   // the empty-box potential, solved once, before any capture
    const pic_status st = ensure_vacuum_potential(c);
    if (st != PIC_OK) return st;
  }
  for (int k = 0; k < 2; ++k)
    for (int v = 0; v < 2; ++v) {
      if (c->gexec[k][v]) cudaGraphExecDestroy(c->gexec[k][v]);
      if (c->graph[k][v]) cudaGraphDestroy(c->graph[k][v]);
      c->gexec[k][v] = nullptr;
      c->graph[k][v] = nullptr;
    }
  for (int k = 0; k < 3; ++k) {
    if (c->gexec_dp[k]) cudaGraphExecDestroy(c->gexec_dp[k]);
    if (c->graph_dp[k]) cudaGraphDestroy(c->graph_dp[k]);
    c->gexec_dp[k] = nullptr;
    c->graph_dp[k] = nullptr;
  }
  c->cfg.warm_start = mode;
  return PIC_OK;
}

pic_status pic_learned_target(pic_ctx *c, int32_t hpad, double scale, float *t) {
  if (!c || !t) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  return learned_target(c, hpad, scale, t);
}

pic_status pic_load(pic_ctx *c, int32_t species, int64_t n, const double *x, const double *y,
                    const double *vx, const double *vy, const uint32_t *ids, uint32_t flags) {
  if (!c) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  const size_t nn = size_t(c->g.nxn) * c->g.nyn;
  if (species == -1) {
    if (!x || n != int64_t(nn)) return PIC_EINVAL;
    const std::vector<float2> xp = to_pairs(x, nn);
    if (cudaMemcpyAsync(c->d_rho_ext, xp.data(), nn * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return PIC_ECUDA;
    c->fields_dirty = 1;
    return check(cudaStreamSynchronize(c->stream));
  }
  if (species == -2) {
    // the potential (initial guess of the next solve); Dirichlet nodes keep their values
    if (!x || n != int64_t(nn)) return PIC_EINVAL;
    std::vector<double> phi(x, x + nn);
    for (size_t k = 0; k < nn; ++k)
      if (!(c->h_nodeflags[k] & kFree)) phi[k] = c->h_g[k];
    const std::vector<float2> pp = to_pairs(phi.data(), nn);
    if (cudaMemcpyAsync(c->d_phi, pp.data(), nn * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return PIC_ECUDA;
    return check(cudaStreamSynchronize(c->stream));
  }
  if (species < 0 || species > 1 || n < 0) return PIC_EINVAL;
  if (n > 0 && (!x || !y || !vx || !vy)) return PIC_EINVAL;
  if (n > c->cfg.capacity[species]) return PIC_EOVERFLOW;
  const int s = species;
  // pinned host arrays the device can address are read by the conversion
  // kernel in place (one launch, no staging copies); others go through the
  // device staging buffer
  auto device_view = [](const void *p) -> const void * {
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  };
  const void *hx = device_view(x), *hy = device_view(y), *hvx = device_view(vx), *hvy = device_view(vy);
  const void *hid = ids ? device_view(ids) : nullptr;
  const bool direct = n > 0 && hx && hy && hvx && hvy && (!ids || hid);
  if (direct &&
      launch_load_convert(c, s, static_cast<const double *>(hx), static_cast<const double *>(hy),
                          static_cast<const double *>(hvx), static_cast<const double *>(hvy),
                          static_cast<const uint32_t *>(hid), 0, n) != cudaSuccess)
    return PIC_ECUDA;
  double *sx = c->d_stage, *sy = sx + c->stage_n, *svx = sy + c->stage_n, *svy = svx + c->stage_n;
  uint32_t *sid = (uint32_t *)(svy + c->stage_n);
  for (int64_t off = 0; !direct && off < n; off += c->stage_n) {
    const int64_t m = std::min<int64_t>(c->stage_n, n - off);
    cudaMemcpyAsync(sx, x + off, m * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(sy, y + off, m * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(svx, vx + off, m * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(svy, vy + off, m * 8, cudaMemcpyHostToDevice, c->stream);
    if (ids) cudaMemcpyAsync(sid, ids + off, m * 4, cudaMemcpyHostToDevice, c->stream);
    cudaError_t e = launch_load_convert(c, s, sx, sy, svx, svy, ids ? sid : nullptr, off, m);
    if (e != cudaSuccess) return PIC_ECUDA;
  }
  int64_t slots[1] = {n};
  cudaMemcpyAsync(c->d_nslots + s, slots, 8, cudaMemcpyHostToDevice, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return PIC_ECUDA;
  c->pending_kick[s] = (flags & PIC_LOAD_V_AT_T0) ? 1 : 0;
  c->fields_dirty = 1;
  c->needs_sort = 1;
  return PIC_OK;
}

pic_status pic_step(pic_ctx *c, int32_t nsteps) {
  if (!c || nsteps < 0) return PIC_EINVAL;
  if (c->cfg.decomposed) return PIC_ESTATE;   // steps of a decomposed run come in two phases
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  pic_status st = prepare(c);
  if (st != PIC_OK) return st;
  for (int32_t k = 0; k < nsteps; ++k) {
    // the interval in force: fixed, or tuned (a sort opens the measurement,
    // none during it, then the chosen interval)
    const bool tuning = c->cfg.sort_every == 0 && c->tune_state < 2;
    bool sorting;
    if (c->cfg.sort_every > 0) sorting = c->steps_since_sort >= c->cfg.sort_every;
    else if (c->tune_state == 0) sorting = true;
    else if (c->tune_state == 1) sorting = false;
    else sorting = c->steps_since_sort >= c->sort_interval;
    if (c->suppress_sort) sorting = false;
    // particles restored from a checkpoint, or a new tile variant, are sorted before they move
    if (c->needs_sort) sorting = true;
    c->needs_sort = 0;
    // steps of the host loop are always timed; graph steps when timing is on
    // or the sort interval is being tuned
    const bool timed = c->cfg.timing || tuning || !c->cfg.graphs;
    if (timed && !c->tpool[0][0]) {
      for (int s = 0; s < kTimeSlots; ++s)
        for (int q = 0; q < kPhaseEvents; ++q)
          if (cudaEventCreate(&c->tpool[s][q]) != cudaSuccess) return PIC_ECUDA;
    }
    const int slot = c->tpend;
    if (c->cfg.graphs) {
      const int ws = sorting ? 1 : 0, ev = timed ? 1 : 0;
      if ((st = check(step_graph(c, ws, ev))) != PIC_OK) return st;
      if (timed) {
        for (int q = 0; q < kPhaseEvents; ++q)
          if (note(cudaGraphExecEventRecordNodeSetEvent(c->gexec[ws][1], c->evnode[ws][q], c->tpool[slot][q]),
                   "step graph event") != cudaSuccess)
            return PIC_ECUDA;
      }
      // particle kernel, [sort], [density]; the solve's kernels are counted from its totals
      c->launches += (sorting ? 4 : 0) + (rho_in_solve(c) ? 1 : 2) +
                     (c->cfg.phi_rf_amp != 0.0 && (c->n_rf_dir || c->n_rf_lift) ? 1 : 0);
      if (note(cudaGraphLaunch(c->gexec[ws][ev], c->stream), "step graph launch") != cudaSuccess)
        return PIC_ECUDA;
      if (sorting) {
        c->cur[0] ^= 1;   // mirror the device-side buffer flip of the sort
        c->cur[1] ^= 1;
      }
    } else {
      if ((st = step_kernels(c, sorting, c->tpool[slot])) != PIC_OK) return st;
    }
    if (sorting) {
      c->steps_since_sort = 0;
      c->t_sorts += 1;
    }
    c->steps_since_sort += 1;
    c->step += 1;
    c->t_steps += 1;
    if (timed) {
      c->tslot_tune[slot] = tuning ? 1 : 0;
      c->tpend += 1;
      // the tuning decides the next step's sort: read its slot now
      if (tuning || !c->cfg.graphs || c->tpend == kTimeSlots)
        if ((st = flush_timing(c)) != PIC_OK) return st;
    }
  }
  return PIC_OK;
}

namespace picgb {
namespace {

// graph of one phase of a decomposed step (k: 0 particles, 1 particles with
// the sort, 2 fields), captured once
cudaError_t phase_graph(pic_ctx *c, int k) {
  if (c->gexec_dp[k]) return cudaSuccess;
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> deps;
  e = note(capture_step(c, g, deps, k == 1 ? 1 : 0, false, k == 2 ? 2 : 1), "phase graph capture");
  if (e == cudaSuccess) e = note(cudaGraphInstantiate(&c->gexec_dp[k], g, 0), "phase graph instantiate");
  if (e == cudaSuccess) c->graph_dp[k] = g;
  else cudaGraphDestroy(g);
  cudaGetLastError();
  return e;
}

__global__ void k_exchange_sum(DevPtrs p, int n, long long count) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    unsigned long long s = 0;
    for (int r = 0; r < n; ++r) s += p.p[r][k];
    for (int r = 0; r < n; ++r) p.p[r][k] = s;
  }
}

}  // namespace
}  // namespace picgb

pic_status pic_step_particles(pic_ctx *c) {
  if (!c || !c->cfg.decomposed) return PIC_EINVAL;
  if (c->phase != 0) return PIC_ESTATE;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  const size_t nn = size_t(c->g.nxn) * c->g.nyn;
  pic_status st;
  if (c->fields_dirty) {
    // bring the fields up to date: deposit of the loaded particles
    if ((st = check(launch_sort(c))) != PIC_OK) return st;
    c->steps_since_sort = 0;
    c->needs_sort = 0;
    if ((st = check(launch_particles(c, 1, 0.f, nullptr))) != PIC_OK) return st;
    if (cudaMemcpyAsync(c->d_acc + 2 * nn, c->d_bottom, 2 * size_t(c->g.ny) * 8, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      return PIC_ECUDA;
    c->phase = 1;
    return PIC_OK;
  }
  const bool sorting = c->steps_since_sort >= c->cfg.sort_every || c->needs_sort;
  c->needs_sort = 0;
  if (c->cfg.graphs) {
    if ((st = check(phase_graph(c, sorting ? 1 : 0))) != PIC_OK) return st;
    if (note(cudaGraphLaunch(c->gexec_dp[sorting ? 1 : 0], c->stream), "phase graph launch") != cudaSuccess)
      return PIC_ECUDA;
    if (sorting) {
      c->cur[0] ^= 1;
      c->cur[1] ^= 1;
    }
    c->launches += (sorting ? 4 : 0) + 1;
  } else {
    if (sorting && (st = check(launch_sort(c))) != PIC_OK) return st;
    if ((st = check(launch_particles(c, 0, 1.f, nullptr))) != PIC_OK) return st;
    if (cudaMemcpyAsync(c->d_acc + 2 * nn, c->d_bottom, 2 * size_t(c->g.ny) * 8, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      return PIC_ECUDA;
    c->launches += (sorting ? 4 : 0) + 1;
  }
  if (sorting) {
    c->steps_since_sort = 0;
    c->t_sorts += 1;
  }
  c->steps_since_sort += 1;
  c->phase = 2;
  return PIC_OK;
}

pic_status pic_step_fields(pic_ctx *c) {
  if (!c || !c->cfg.decomposed) return PIC_EINVAL;
  if (c->phase == 0) return PIC_ESTATE;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  pic_status st;
  if (c->phase == 1) {
    // the rest of the bring-up: rho, a cold solve, pending half kicks
    c->phase = 0;
    if ((st = check(launch_rf_bias(c, 0))) != PIC_OK) return st;
    if ((st = check(launch_rho(c, 0))) != PIC_OK) return st;
    if ((st = poisson_solve(c, true)) != PIC_OK) return st;
    if (cudaMemcpyAsync(c->d_phi_prev, c->d_phi, size_t(c->g.nxn) * c->g.nyn * sizeof(float2),
                        cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      return PIC_ECUDA;
    if (c->pending_kick[0] || c->pending_kick[1]) {
      if ((st = check(launch_particles(c, 2, -0.5f, c->pending_kick))) != PIC_OK) return st;
      c->pending_kick[0] = c->pending_kick[1] = 0;
    }
    c->fields_dirty = 0;
    return PIC_OK;
  }
  c->phase = 0;
  if (c->cfg.graphs) {
    if ((st = check(phase_graph(c, 2))) != PIC_OK) return st;
    if (note(cudaGraphLaunch(c->gexec_dp[2], c->stream), "phase graph launch") != cudaSuccess) return PIC_ECUDA;
    c->launches += (rho_in_solve(c) ? 0 : 1) +
                   (c->cfg.phi_rf_amp != 0.0 && (c->n_rf_dir || c->n_rf_lift) ? 1 : 0);
  } else {
    if ((st = check(launch_rf_bias(c, 1))) != PIC_OK) return st;
    if ((st = check(launch_rho(c, 1))) != PIC_OK) return st;
    if ((st = poisson_solve(c, c->cfg.warm_start == 0)) != PIC_OK) return st;
    c->launches += 1;
  }
  c->step += 1;
  c->t_steps += 1;
  return PIC_OK;
}

pic_status pic_exchange_buffer(pic_ctx *c, int64_t **buf, int64_t *count) {
  if (!c || !buf || !count) return PIC_EINVAL;
  *buf = reinterpret_cast<int64_t *>(c->d_acc);
  *count = 2 * int64_t(c->g.nxn) * c->g.nyn + 2 * int64_t(c->g.ny);
  return PIC_OK;
}

pic_status pic_exchange_sum(pic_ctx *const *ctxs, int32_t n) {
  if (!ctxs || n < 1 || n > 64) return PIC_EINVAL;
  DevPtrs p = {};
  int64_t count = -1;
  for (int32_t r = 0; r < n; ++r) {
    pic_ctx *c = ctxs[r];
    if (!c || !c->cfg.decomposed || c->dev != ctxs[0]->dev || c->phase == 0) return PIC_EINVAL;
    int64_t *b, m;
    pic_exchange_buffer(c, &b, &m);
    if (count >= 0 && m != count) return PIC_EINVAL;
    count = m;
    p.p[r] = reinterpret_cast<unsigned long long *>(b);
    if (cudaSetDevice(c->dev) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
      return PIC_ECUDA;
  }
  cudaStream_t s = ctxs[0]->stream;
  k_exchange_sum<<<ctxs[0]->num_sms * 4, 256, 0, s>>>(p, n, (long long)count);
  if (note(cudaGetLastError(), "exchange sum") != cudaSuccess) return PIC_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

namespace picgb {
namespace {

void drop_step_graphs(pic_ctx *c) {
  for (int k = 0; k < 2; ++k)
    for (int v = 0; v < 2; ++v) {
      if (c->gexec[k][v]) cudaGraphExecDestroy(c->gexec[k][v]);
      if (c->graph[k][v]) cudaGraphDestroy(c->graph[k][v]);
      c->gexec[k][v] = nullptr;
      c->graph[k][v] = nullptr;
    }
  for (int k = 0; k < 3; ++k) {
    if (c->gexec_dp[k]) cudaGraphExecDestroy(c->gexec_dp[k]);
    if (c->graph_dp[k]) cudaGraphDestroy(c->graph_dp[k]);
    c->gexec_dp[k] = nullptr;
    c->graph_dp[k] = nullptr;
  }
}

// Key of a tuning-cache entry: the GPU, the grid and geometry, the loading.
std::string tune_key(pic_ctx *c) {
  cudaDeviceProp prop;
  std::string gpu = "unknown";
  if (cudaGetDeviceProperties(&prop, c->dev) == cudaSuccess) gpu = prop.name;
  for (char &ch : gpu)
    if (ch == '"' || ch == '|' || ch == '\\') ch = '_';
  const pic_config &f = c->cfg;
  return gpu + "|" + std::to_string(f.nx) + "|" + std::to_string(f.ny) + "|" + std::to_string(f.periodic_x) +
         "|" + std::to_string(f.periodic_y) + "|" + std::to_string(f.trench_depth) + "|" +
         std::to_string(f.trench_width) + "|" + std::to_string(f.ppc[0]) + "|" + std::to_string(f.ppc[1]);
}

// The cache is a JSON array with one object per line; the entry of a key is
// the line holding "key": "<key>", its choice the value of "tile_variant".
int cache_lookup(const char *path, const std::string &key) {
  std::FILE *f = std::fopen(path, "r");
  if (!f) return -1;
  const std::string want = "\"key\": \"" + key + "\"";
  char line[4096];
  int found = -1;
  while (std::fgets(line, sizeof(line), f)) {
    const std::string l(line);
    if (l.find(want) == std::string::npos) continue;
    const size_t p = l.find("\"tile_variant\": ");
    if (p != std::string::npos) found = std::atoi(l.c_str() + p + 16);
  }
  std::fclose(f);
  return (found >= 0 && found < kNumTileVariants) ? found : -1;
}

bool cache_store(const char *path, const std::string &key, int v, const double *ms) {
  std::vector<std::string> keep;
  if (std::FILE *f = std::fopen(path, "r")) {
    char line[4096];
    const std::string want = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof(line), f)) {
      std::string l(line);
      while (!l.empty() && (l.back() == '\n' || l.back() == ',')) l.pop_back();
      if (l.size() > 1 && l[0] == '{' && l.find(want) == std::string::npos) keep.push_back(l);
    }
    std::fclose(f);
  }
  char buf[1024];
  std::snprintf(buf, sizeof(buf),
                "{\"key\": \"%s\", \"tile_variant\": %d, \"particle_ms\": [%.5f, %.5f, %.5f, %.5f]}",
                key.c_str(), v, ms[0], ms[1], ms[2], ms[3]);
  keep.push_back(buf);
  const std::string tmp = std::string(path) + ".tmp";
  std::FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fputs("[\n", f);
  for (size_t k = 0; k < keep.size(); ++k) {
    std::fputs(keep[k].c_str(), f);
    std::fputs(k + 1 < keep.size() ? ",\n" : "\n", f);
  }
  std::fputs("]\n", f);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

}  // namespace
}  // namespace picgb

pic_status pic_autotune(pic_ctx *c, int32_t steps, const char *cache_path, int32_t *chosen) {
  if (!c || steps < 1 || c->cfg.decomposed) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  const std::string key = tune_key(c);
  int best = cache_path ? cache_lookup(cache_path, key) : -1;
  double ms[kNumTileVariants] = {0, 0, 0, 0};
  pic_status st = PIC_OK;
  if (best < 0) {
    // time the particle kernel of each variant over `steps` steps right after
    // its own sort (no scheduled sort in between); the steps advance the run,
    // whose results do not depend on the variant
    st = pic_step(c, 0);
    const int timing_save = c->cfg.timing;
    double best_ms = 0.0;
    for (int v = 0; v < kNumTileVariants && st == PIC_OK; ++v) {
      drop_step_graphs(c);
      set_tile_variant(c, v);
      if ((st = pic_step(c, 1)) != PIC_OK) break;   // sorts into the new tiles
      c->cfg.timing = 1;
      c->suppress_sort = 1;
      if ((st = flush_timing(c)) != PIC_OK) break;
      const double p0 = c->t_part;
      const int64_t n0 = c->t_steps;
      st = pic_step(c, steps);
      if (st == PIC_OK) st = flush_timing(c);
      c->suppress_sort = 0;
      c->cfg.timing = timing_save;
      ms[v] = (c->t_part - p0) / double(std::max<int64_t>(c->t_steps - n0, 1));
      if (best < 0 || ms[v] < best_ms) {
        best = v;
        best_ms = ms[v];
      }
    }
    c->suppress_sort = 0;
    c->cfg.timing = timing_save;
    if (st != PIC_OK) return st;
    if (cache_path && !cache_store(cache_path, key, best, ms)) st = PIC_EINVAL;
  }
  drop_step_graphs(c);
  set_tile_variant(c, best);
  c->cfg.tile_variant = best;
  // a tuned sort interval is chosen again for the new tiles
  if (c->cfg.sort_every == 0) c->tune_state = 0;
  if (chosen) *chosen = best;
  return st;
}

pic_status pic_set_timing(pic_ctx *c, int32_t on) {
  if (!c || on < 0 || on > 1) return PIC_EINVAL;
  c->cfg.timing = on;
  return PIC_OK;
}

pic_status pic_diag(pic_ctx *c, int32_t kind, void *out, int64_t cap_bytes, int64_t *n_out) {
  if (!c || (!out && kind != PIC_DIAG_STATUS)) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  if (flush_timing(c) != PIC_OK || count_solves(c) != PIC_OK) return PIC_ECUDA;
  const Geom &g = c->g;
  const size_t nn = size_t(g.nxn) * g.nyn;
  int64_t count = 0;
  auto need = [&](int64_t bytes) { return bytes <= cap_bytes; };
  uint32_t bits = 0;
  if (cudaMemcpy(&bits, c->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  auto species_moments = [&](double m[2][3]) -> pic_status {
    const int nb = c->num_sms * 2;
    double *d = c->d_diag;
    for (int s = 0; s < 2; ++s) {
      if (launch_moments(c, s, d + s * 3 * nb, nb) != cudaSuccess) return PIC_ECUDA;
    }
    std::vector<double> h(2 * 3 * nb);
    if (cudaMemcpyAsync(h.data(), d, h.size() * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return PIC_ECUDA;
    for (int s = 0; s < 2; ++s)
      for (int k = 0; k < 3; ++k) {
        double t = 0;
        for (int b = 0; b < nb; ++b) t += h[(s * nb + b) * 3 + k];
        m[s][k] = t;
      }
    return PIC_OK;
  };
  switch (kind) {
    case PIC_DIAG_ENERGY: {
      if (!need(4 * 8)) return PIC_EINVAL;
      int32_t nch = 0;
      cudaMemcpy(&nch, c->d_nchunks, 4, cudaMemcpyDeviceToHost);
      std::vector<double> ke(std::max(nch, 1));
      std::vector<Chunk> ch(std::max(nch, 1));
      cudaMemcpy(ke.data(), c->d_ke_part, size_t(nch) * 8, cudaMemcpyDeviceToHost);
      cudaMemcpy(ch.data(), c->d_chunks, size_t(nch) * sizeof(Chunk), cudaMemcpyDeviceToHost);
      double fe[2];
      cudaMemcpy(fe, c->d_fe, 16, cudaMemcpyDeviceToHost);
      double kes[2] = {0, 0};
      for (int k = 0; k < nch; ++k) kes[ch[k].species] += ke[k];
      double *o = (double *)out;
      for (int s = 0; s < 2; ++s) {
        const double m = c->cfg.charge[s] / c->cfg.alpha[s];
        o[s] = 0.5 * m * kes[s] / double(c->cfg.ppc[s]);
      }
      o[2] = fe[1];
      o[3] = double(c->step - 1);
      count = 4;
      break;
    }
    case PIC_DIAG_MOMENTUM: {
      if (!need(4 * 8)) return PIC_EINVAL;
      double m[2][3];
      pic_status st = species_moments(m);
      if (st != PIC_OK) return st;
      double *o = (double *)out;
      for (int s = 0; s < 2; ++s) {
        const double mw = c->cfg.charge[s] / c->cfg.alpha[s] / double(c->cfg.ppc[s]);
        o[2 * s] = mw * m[s][0];
        o[2 * s + 1] = mw * m[s][1];
      }
      count = 4;
      break;
    }
    case PIC_DIAG_COUNTS: {
      if (!need(18 * 8)) return PIC_EINVAL;
      double m[2][3];
      pic_status st = species_moments(m);
      if (st != PIC_OK) return st;
      unsigned long long w[2 * PIC_NWALLS];
      cudaMemcpy(w, c->d_walls, sizeof(w), cudaMemcpyDeviceToHost);
      int64_t *o = (int64_t *)out;
      for (int k = 0; k < 2 * PIC_NWALLS; ++k) o[k] = int64_t(w[k]);
      o[16] = int64_t(m[0][2]);
      o[17] = int64_t(m[1][2]);
      count = 18;
      break;
    }
    case PIC_DIAG_SURFACE: {
      if (!need(2 * int64_t(g.ny) * 8)) return PIC_EINVAL;
      cudaMemcpy(out, c->d_bottom, 2 * size_t(g.ny) * 8, cudaMemcpyDeviceToHost);
      count = 2 * g.ny;
      break;
    }
    case PIC_DIAG_HITS: {
      unsigned long long nh = 0;
      cudaMemcpy(&nh, c->d_nhits, 8, cudaMemcpyDeviceToHost);
      int64_t m = std::min<int64_t>(int64_t(nh), c->cfg.hit_capacity);
      m = std::min<int64_t>(m, cap_bytes / int64_t(sizeof(pic_hit)));
      if (m > 0) cudaMemcpy(out, c->d_hits, size_t(m) * sizeof(pic_hit), cudaMemcpyDeviceToHost);
      count = m;
      break;
    }
    case PIC_DIAG_RHO:
    case PIC_DIAG_PHI: {
      if (!need(int64_t(nn) * 8)) return PIC_EINVAL;
      from_pairs(kind == PIC_DIAG_RHO ? c->d_rho : c->d_phi, nn, static_cast<double *>(out));
      count = int64_t(nn);
      break;
    }
    case PIC_DIAG_E: {
      if (!need(2 * int64_t(nn) * 8)) return PIC_EINVAL;
      std::vector<float2> e(nn);
      cudaMemcpy(e.data(), c->d_E, nn * sizeof(float2), cudaMemcpyDeviceToHost);
      double *o = (double *)out;
      for (size_t n = 0; n < nn; ++n) {
        o[n] = e[n].x;
        o[nn + n] = e[n].y;
      }
      count = 2 * int64_t(nn);
      break;
    }
    case PIC_DIAG_STATE_E:
    case PIC_DIAG_STATE_I: {
      const int s = kind == PIC_DIAG_STATE_E ? 0 : 1;
      double m[2][3];
      pic_status st = species_moments(m);
      if (st != PIC_OK) return st;
      const int64_t live = int64_t(m[s][2]);
      if (!need(5 * live * 8)) return PIC_EINVAL;
      // pinned host memory the device can address is written by the export
      // kernel in place; otherwise through a device buffer and one copy
      // (temporaries through the context's allocator)
      double *direct = nullptr;
      {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost)
          direct = static_cast<double *>(at.devicePointer);
        else
          cudaGetLastError();
      }
      double *buf = direct ? nullptr : (double *)tmp_alloc(c, size_t(std::max<int64_t>(live, 1)) * 5 * 8);
      unsigned long long *ctr = (unsigned long long *)tmp_alloc(c, 8);
      if ((!direct && !buf) || !ctr) {
        tmp_free(c, buf);
        tmp_free(c, ctr);
        return PIC_ENOMEM;
      }
      cudaMemsetAsync(ctr, 0, 8, c->stream);
      cudaError_t e = launch_export_state(c, s, direct ? direct : buf, live, ctr);
      if (e == cudaSuccess && !direct)
        e = cudaMemcpyAsync(out, buf, size_t(live) * 5 * 8, cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      tmp_free(c, buf);
      tmp_free(c, ctr);
      if (e != cudaSuccess) return PIC_ECUDA;
      count = live;
      break;
    }
    case PIC_DIAG_POISSON: {
      if (!need(4 * 8)) return PIC_EINVAL;
      PoissonState ps;
      cudaMemcpy(&ps, c->d_ps, sizeof(ps), cudaMemcpyDeviceToHost);
      double *o = (double *)out;
      o[0] = ps.total_iters;
      o[1] = c->last_outer;
      o[2] = ps.rel;
      o[3] = c->last_ms;
      count = 4;
      if (need(5 * 8)) {
        o[4] = ps.rel_first;
        count = 5;
      }
      break;
    }
    case PIC_DIAG_SORT: {
      if (!need(8)) return PIC_EINVAL;
      int32_t *o = (int32_t *)out;
      if (c->cfg.sort_every > 0) {
        o[0] = c->cfg.sort_every;
        o[1] = 0;
      } else {
        o[0] = c->tune_state == 2 ? c->sort_interval : 0;
        o[1] = c->tune_state == 2 ? 1 : 0;
      }
      count = 2;
      break;
    }
    case PIC_DIAG_TILE: {
      if (!need(5 * 4)) return PIC_EINVAL;
      int32_t *o = (int32_t *)out;
      const TileVariant &t = kTileVariants[c->tile_variant];
      o[0] = c->tile_variant;
      o[1] = 1 << t.log2x;
      o[2] = 1 << t.log2y;
      o[3] = t.halo;
      o[4] = t.threads;
      count = 5;
      break;
    }
    case PIC_DIAG_SOLVER: {
      if (!need(4)) return PIC_EINVAL;
      *(int32_t *)out = c->fp.enabled ? 0 : 1;
      count = 1;
      break;
    }
    case PIC_DIAG_PHI_VACUUM: {
      if (!need(int64_t(nn) * 8)) return PIC_EINVAL;
      const pic_status st = ensure_vacuum_potential(c);
      if (st != PIC_OK) return st;
      from_pairs(c->d_phiL, nn, static_cast<double *>(out));
      count = int64_t(nn);
      break;
    }
    case PIC_DIAG_TIMING: {
      if (!need(8 * 8)) return PIC_EINVAL;
      int64_t slots[2] = {0, 0};
      cudaMemcpy(slots, c->d_nslots, 16, cudaMemcpyDeviceToHost);
      double *o = (double *)out;
      o[0] = double(c->t_steps);
      o[1] = c->t_part;
      o[2] = c->t_sort;
      o[3] = c->t_poisson;
      o[4] = c->t_other;
      o[5] = double(c->t_sorts);
      o[6] = double(c->launches);
      o[7] = double(slots[0] + slots[1]);
      c->t_part = c->t_sort = c->t_poisson = c->t_other = 0.0;
      c->t_steps = c->t_sorts = c->launches = 0;
      count = 8;
      break;
    }
    case PIC_DIAG_STATUS: {
      if (out) {
        if (!need(4)) return PIC_EINVAL;
        *(uint32_t *)out = bits;
      }
      cudaMemsetAsync(c->d_status, 0, 4, c->stream);
      count = 1;
      if (n_out) *n_out = count;
      return cudaStreamSynchronize(c->stream) == cudaSuccess ? PIC_OK : PIC_ECUDA;
    }
    default:
      return PIC_EINVAL;
  }
  if (n_out) *n_out = count;
  if (cudaGetLastError() != cudaSuccess) return PIC_ECUDA;
  return status_from_bits(bits);
}

namespace {

// Checkpoint layout (host memory): the header, then per species the live
// particles in stored form (cell, fx, fy, vx, vy, id arrays), the node
// arrays (phi, phi of the previous step, E, rho, rho_ext, Dirichlet data as
// double-float pairs; the lift), the wall and bottom tallies, the hit
// records kept, and the solver's device scalars.
struct CkptHeader {
  char magic[8];
  int32_t version;
  int32_t nx, ny, px, py, nxn, nyn;
  int32_t d_step;
  int64_t n_live[2];
  int64_t hits_kept, hits_total;
  int64_t step;
  uint32_t status;
  int32_t pending_kick[2];
  int32_t reserved;
  double fe[2];
};
constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'G', 'B', 'C', 'K', '1'};

int64_t ckpt_bytes(const pic_ctx *c, const int64_t n_live[2], int64_t hits) {
  const int64_t nn = int64_t(c->g.nxn) * c->g.nyn;
  return int64_t(sizeof(CkptHeader)) + 24 * (n_live[0] + n_live[1]) + nn * (6 * 8 + 4) +
         8 * (2 * PIC_NWALLS + 2 * int64_t(c->g.ny)) + hits * int64_t(sizeof(pic_hit)) +
         int64_t(sizeof(PoissonState));
}

// the node arrays of a checkpoint, in order, with their element sizes
struct NodeArray {
  void *d;
  size_t elem;
};
std::vector<NodeArray> node_arrays(pic_ctx *c) {
  return {{c->d_phi, 8}, {c->d_phi_prev, 8}, {c->d_E, 8}, {c->d_rho, 8},
          {c->d_rho_ext, 8}, {c->d_g, 8}, {c->d_lift, 4}};
}

}  // namespace

pic_status pic_save(pic_ctx *c, void *buf, int64_t cap_bytes, int64_t *n_out) {
  if (!c) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  if (c->fields_dirty) return PIC_ESTATE;   // loaded but not yet brought up to date
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  int64_t nslots[2];
  unsigned long long nh = 0;
  if (cudaMemcpy(nslots, c->d_nslots, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&nh, c->d_nhits, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PIC_ECUDA;
  // live counts: compaction of each species into a temporary device buffer
  ParticleBuf tmp[2] = {};
  void *mem[2] = {nullptr, nullptr};
  unsigned long long *ctr = (unsigned long long *)tmp_alloc(c, 16);
  pic_status st = ctr ? PIC_OK : PIC_ENOMEM;
  int64_t n_live[2] = {0, 0};
  for (int s = 0; s < 2 && st == PIC_OK; ++s) {
    const int64_t m = std::max<int64_t>(nslots[s], 1);
    mem[s] = tmp_alloc(c, size_t(m) * 24);
    if (!mem[s]) {
      st = PIC_ENOMEM;
      break;
    }
    char *b = (char *)mem[s];
    tmp[s] = ParticleBuf{(int32_t *)b, (float *)(b + 4 * m), (float *)(b + 8 * m),
                         (float *)(b + 12 * m), (float *)(b + 16 * m), (uint32_t *)(b + 20 * m)};
    cudaMemsetAsync(ctr + s, 0, 8, c->stream);
    if (launch_export_raw(c, s, tmp[s], m, ctr + s) != cudaSuccess) st = PIC_ECUDA;
  }
  unsigned long long cnt[2] = {0, 0};
  if (st == PIC_OK && (cudaMemcpyAsync(cnt, ctr, 16, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                       cudaStreamSynchronize(c->stream) != cudaSuccess))
    st = PIC_ECUDA;
  n_live[0] = int64_t(cnt[0]);
  n_live[1] = int64_t(cnt[1]);
  const int64_t hits = std::min<int64_t>(int64_t(nh), c->cfg.hit_capacity);
  const int64_t bytes = ckpt_bytes(c, n_live, hits);
  if (n_out) *n_out = bytes;
  if (st == PIC_OK && buf && cap_bytes < bytes) st = PIC_EINVAL;
  if (st == PIC_OK && buf) {
    char *o = (char *)buf;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.nx = c->g.nx;
    h.ny = c->g.ny;
    h.px = c->g.px;
    h.py = c->g.py;
    h.nxn = c->g.nxn;
    h.nyn = c->g.nyn;
    h.n_live[0] = n_live[0];
    h.n_live[1] = n_live[1];
    h.hits_kept = hits;
    h.hits_total = int64_t(nh);
    h.step = c->step;
    h.pending_kick[0] = c->pending_kick[0];
    h.pending_kick[1] = c->pending_kick[1];
    cudaError_t e = cudaMemcpy(&h.d_step, c->d_step, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h.status, c->d_status, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h.fe, c->d_fe, 16, cudaMemcpyDeviceToHost);
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      const int64_t m = std::max<int64_t>(nslots[s], 1), n = n_live[s];
      // the six arrays of the compacted buffer, n elements each
      for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
        e = cudaMemcpy(o, (char *)mem[s] + 4 * k * m, size_t(n) * 4, cudaMemcpyDeviceToHost);
        o += 4 * n;
      }
    }
    const size_t nn = size_t(c->g.nxn) * c->g.nyn;
    for (const NodeArray &a : node_arrays(c)) {
      if (e == cudaSuccess) e = cudaMemcpy(o, a.d, nn * a.elem, cudaMemcpyDeviceToHost);
      o += nn * a.elem;
    }
    if (e == cudaSuccess) e = cudaMemcpy(o, c->d_walls, 8 * 2 * PIC_NWALLS, cudaMemcpyDeviceToHost);
    o += 8 * 2 * PIC_NWALLS;
    if (e == cudaSuccess) e = cudaMemcpy(o, c->d_bottom, 8 * 2 * size_t(c->g.ny), cudaMemcpyDeviceToHost);
    o += 8 * 2 * size_t(c->g.ny);
    if (e == cudaSuccess && hits > 0) e = cudaMemcpy(o, c->d_hits, size_t(hits) * sizeof(pic_hit), cudaMemcpyDeviceToHost);
    o += size_t(hits) * sizeof(pic_hit);
    if (e == cudaSuccess) e = cudaMemcpy(o, c->d_ps, sizeof(PoissonState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = PIC_ECUDA;
  }
  for (int s = 0; s < 2; ++s) tmp_free(c, mem[s]);
  tmp_free(c, ctr);
  return st;
}

pic_status pic_restore(pic_ctx *c, const void *buf, int64_t n_bytes) {
  if (!c || !buf || n_bytes < int64_t(sizeof(CkptHeader))) return PIC_EINVAL;
  if (cudaSetDevice(c->dev) != cudaSuccess) return PIC_ECUDA;
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1) return PIC_EINVAL;
  if (h.nx != c->g.nx || h.ny != c->g.ny || h.px != c->g.px || h.py != c->g.py || h.nxn != c->g.nxn ||
      h.nyn != c->g.nyn)
    return PIC_EINVAL;
  for (int s = 0; s < 2; ++s)
    if (h.n_live[s] < 0 || h.n_live[s] > c->cfg.capacity[s]) return PIC_EOVERFLOW;
  if (h.hits_kept < 0 || h.hits_kept > c->cfg.hit_capacity || h.hits_total < h.hits_kept) return PIC_EINVAL;
  if (n_bytes != ckpt_bytes(c, h.n_live, h.hits_kept)) return PIC_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PIC_ECUDA;
  const char *o = (const char *)buf + sizeof(h);
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    const ParticleBuf &P = c->pb[s][c->cur[s]];
    void *dst[6] = {P.cell, P.fx, P.fy, P.vx, P.vy, P.id};
    const int64_t n = h.n_live[s];
    for (int k = 0; k < 6; ++k) {
      if (e == cudaSuccess && n > 0) e = cudaMemcpy(dst[k], o, size_t(n) * 4, cudaMemcpyHostToDevice);
      o += 4 * n;
    }
  }
  const size_t nn = size_t(c->g.nxn) * c->g.nyn;
  for (const NodeArray &a : node_arrays(c)) {
    if (e == cudaSuccess) e = cudaMemcpy(a.d, o, nn * a.elem, cudaMemcpyHostToDevice);
    o += nn * a.elem;
  }
  if (e == cudaSuccess) e = cudaMemcpy(c->d_walls, o, 8 * 2 * PIC_NWALLS, cudaMemcpyHostToDevice);
  o += 8 * 2 * PIC_NWALLS;
  if (e == cudaSuccess) e = cudaMemcpy(c->d_bottom, o, 8 * 2 * size_t(c->g.ny), cudaMemcpyHostToDevice);
  o += 8 * 2 * size_t(c->g.ny);
  if (e == cudaSuccess && h.hits_kept > 0)
    e = cudaMemcpy(c->d_hits, o, size_t(h.hits_kept) * sizeof(pic_hit), cudaMemcpyHostToDevice);
  o += size_t(h.hits_kept) * sizeof(pic_hit);
  // the solver's scalars, keeping this context's running launch totals
  PoissonState ps;
  std::memcpy(&ps, o, sizeof(ps));
  PoissonState mine;
  if (e == cudaSuccess) e = cudaMemcpy(&mine, c->d_ps, sizeof(mine), cudaMemcpyDeviceToHost);
  ps.n_solves = mine.n_solves;
  ps.sum_outer = mine.sum_outer;
  ps.sum_total = mine.sum_total;
  if (e == cudaSuccess) e = cudaMemcpy(c->d_ps, &ps, sizeof(ps), cudaMemcpyHostToDevice);
  const unsigned long long nh = (unsigned long long)h.hits_total;
  const int64_t slots[2] = {h.n_live[0], h.n_live[1]};
  if (e == cudaSuccess) e = cudaMemcpy(c->d_nhits, &nh, 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_nslots, slots, 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_step, &h.d_step, 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_status, &h.status, 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_fe, h.fe, 16, cudaMemcpyHostToDevice);
  // no particle kernel has run on the restored particles: no work items yet
  const int32_t zero = 0;
  if (e == cudaSuccess) e = cudaMemcpy(c->d_nchunks, &zero, 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return PIC_ECUDA;
  c->step = h.step;
  c->pending_kick[0] = h.pending_kick[0];
  c->pending_kick[1] = h.pending_kick[1];
  c->fields_dirty = 0;
  c->needs_sort = 1;
  return PIC_OK;
}

pic_status pic_free(pic_ctx *c) {
  if (!c) return PIC_OK;
  cudaSetDevice(c->dev);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) tmp_free(c, p);
  c->allocs.clear();
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_ps) cudaFreeHost(c->h_ps);
  for (int k = 0; k < 2; ++k)
    for (int v = 0; v < 2; ++v) {
      if (c->gexec[k][v]) cudaGraphExecDestroy(c->gexec[k][v]);
      if (c->graph[k][v]) cudaGraphDestroy(c->graph[k][v]);
    }
  for (int q = 0; q < kPhaseEvents; ++q) {
    if (c->tev[q]) cudaEventDestroy(c->tev[q]);
    for (int s = 0; s < kTimeSlots; ++s)
      if (c->tpool[s][q]) cudaEventDestroy(c->tpool[s][q]);
  }
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->net) pic_unet_free(c->net);
  for (int k = 0; k < 3; ++k) {
    if (c->gexec_dp[k]) cudaGraphExecDestroy(c->gexec_dp[k]);
    if (c->graph_dp[k]) cudaGraphDestroy(c->graph_dp[k]);
  }
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return PIC_OK;
}

}  // extern "C"
