// ensemble_abi.cu -- the ensemble entry points of include/lbmd.h: many
// independent translocation realisations (Sec. III, ensembles over initial
// chains) stepped together.  Every realisation keeps the workspace layout of a
// single box; the ensemble adds the descriptor array, the tile list of the
// stream-collide, the (realisation, bead) table of the gather and
// spread, the chain lists of the MD groups and the live flags.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "lbmd_host.h"

using namespace lbmd;

namespace {

constexpr int kEnsSide = 4;     // side streams for the MD groups
constexpr int kEnsBlock = 16;   // steps per long graph
const int kEnsGraphSteps[3] = {1, 2, kEnsBlock};

struct EnsLayout {
  size_t mem, lbd, tiles, n_tiles, beads, live, cap, chains, stage;
  size_t stage_floats;
  size_t max_tiles;  // tile capacity (rows = 4, every realisation)
  int nb;            // padded bead slots
  std::vector<size_t> off;   // workspace offset of each realisation
  std::vector<Layout> L;
  size_t total;
};

// Tiles of 32 x rows consecutive nodes per z-plane.
size_t tiles_of(const lbmd_params &p, int rows) {
  const size_t plane = (size_t)p.nx * p.ny, ts = (size_t)32 * rows;
  return (plane + ts - 1) / ts * (size_t)p.nz;
}

int validate_members(const lbmd_params *m, int32_t count) {
  if (!m) return fail(LBMD_EINVAL, "members is NULL");
  if (count < 1) return fail(LBMD_EINVAL, "count must be >= 1");
  for (int k = 0; k < count; ++k) {
    int rc = validate(&m[k]);
    if (rc) {
      char buf[512];
      snprintf(buf, sizeof(buf), "%s", last_message());
      return fail(rc, "member %d: %s", k, buf);
    }
    if (m[k].n_beads < 1) return fail(LBMD_EINVAL, "member %d: n_beads must be >= 1", k);
    const long long V = (long long)m[k].nx * m[k].ny * m[k].nz;
    if (19 * ((V + 63) / 64 * 64) >= 0x7fffffffLL)
      return fail(LBMD_EUNSUPPORTED, "member %d: box too large for 32-bit population offsets", k);
    if (m[k].kT_fluid != 0.0)
      return fail(LBMD_EUNSUPPORTED, "member %d: the thermal source is single-box only", k);
    if (m[k].streaming != LBMD_STREAM_PULL)
      return fail(LBMD_EUNSUPPORTED, "member %d: in-place streaming is single-box only", k);
    if ((long long)m[k].nx * m[k].ny >= (1LL << 22))
      return fail(LBMD_EUNSUPPORTED, "member %d: nx * ny must be < 2^22", k);
    if (m[k].storage != m[0].storage || m[k].forcing != m[0].forcing ||
        m[k].solvent_free != m[0].solvent_free)
      return fail(LBMD_EUNSUPPORTED,
                  "member %d: storage, forcing and solvent_free must match member 0", k);
  }
  return LBMD_OK;
}

EnsLayout make_ens_layout(const lbmd_params *m, int32_t count) {
  EnsLayout E;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  E.max_tiles = 0;
  E.nb = 0;
  E.stage_floats = 0;
  for (int k = 0; k < count; ++k) {
    E.max_tiles += tiles_of(m[k], 4);
    E.nb += (m[k].n_beads + 3) / 4 * 4;
    E.stage_floats = std::max(E.stage_floats, stage_floats_for(m[k]));
  }
  E.mem = take((size_t)count * sizeof(EnsMember));
  E.lbd = take((size_t)count * sizeof(EnsLb));
  E.tiles = take(std::max<size_t>(E.max_tiles, 1) * sizeof(EnsTile));
  E.n_tiles = take(sizeof(int));
  E.beads = take((size_t)std::max(E.nb, 1) * sizeof(int2));
  E.live = take(2 * (size_t)count * sizeof(int));
  E.cap = take(sizeof(long long));
  E.chains = take((size_t)count * sizeof(int));
  E.stage = take(E.stage_floats * sizeof(float));
  E.off.resize(count);
  E.L.resize(count);
  for (int k = 0; k < count; ++k) {
    E.L[k] = make_layout(m[k], false);
    E.off[k] = take(E.L[k].total);
  }
  E.total = o;
  return E;
}

struct Group {  // chains sharing one MD block size
  int threads, max_n, first, count;
};

}  // namespace

struct lbmd_ensemble {
  int count, storage, forcing, solvent_free;
  std::vector<lbmd_params> p;  // host pointers cleared
  EnsLayout E;
  char *ws;
  std::vector<Instance> inst;
  std::vector<EnsMember> hmem;
  std::vector<EnsLb> hlbd;
  std::vector<Group> groups;
  EnsMember *d_mem;
  EnsLb *d_lbd;
  EnsTile *d_tiles;
  int *d_n_tiles, *d_live, *d_chains;
  int2 *d_beads;
  long long *d_cap;
  float *stage;
  int rows, warps, claim, cpt, grid, sms;
  long long G;        // ensemble steps enqueued so far
  long long cap;
  int tiles_live;     // realisations in the current tile list
  std::vector<EnsTile> htiles;
  cudaStream_t user, own, side[kEnsSide];
  int nside, prio_high;
  cudaEvent_t ev_in, ev_out, ev_fork, ev_join[kEnsSide];
  cudaGraphExec_t graph[2][3];
  int timing;
  std::vector<cudaEvent_t> tev;  // per timed step: step start, lb start, lb end, step end
  size_t tev_used;
  double timed_lb, timed_step;
  long long timed_count;
  int sticky;
};

namespace {

int ens_fail(lbmd_ensemble *e, cudaError_t err, const char *what) {
  if (e) e->sticky = LBMD_ECUDA;
  return fail(LBMD_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}
#define EK(ens, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ens_fail(ens, e_, #call);  \
  } while (0)

int check_ens(lbmd_ensemble *e) {
  if (!e) return fail(LBMD_EINVAL, "ensemble is NULL");
  if (e->sticky) return e->sticky;
  return LBMD_OK;
}

void drop_graphs(lbmd_ensemble *e) {
  for (auto &row : e->graph)
    for (auto &gx : row)
      if (gx) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
}

// Two x-adjacent nodes per thread need 16-bit storage and even rows.
bool xpair_ok(const lbmd_ensemble *e) {
  if (e->storage == LBMD_STORE_F32) return false;
  for (const lbmd_params &p : e->p)
    if (p.nx % 2) return false;
  return true;
}

// Tile list of the realisations flagged in `live` for the current tile
// height, uploaded on the private stream (synchronised before the host
// vector can change again).
cudaError_t upload_tiles(lbmd_ensemble *e, const std::vector<int> &live) {
  e->htiles.clear();
  int n_live = 0;
  for (int m = 0; m < e->count; ++m) {
    if (!live[m]) continue;
    ++n_live;
    const lbmd_params &p = e->p[m];
    // nodes per tile: 32 x rows (64 x rows for x-pairs), one plane (two for
    // z-pairs)
    const int plane = p.nx * p.ny, ts = (e->cpt == kEnsXPair ? 64 : 32) * e->rows;
    const int dz = e->cpt == 2 ? 2 : 1;
    for (int z0 = 0; z0 < p.nz; z0 += dz)
      for (int r0 = 0; r0 < plane; r0 += ts)
        e->htiles.push_back(EnsTile{m, z0, r0, std::min(dz, p.nz - z0)});
  }
  const int n = (int)e->htiles.size();
  cudaError_t err;
  if (n > 0 &&
      (err = cudaMemcpyAsync(e->d_tiles, e->htiles.data(), n * sizeof(EnsTile), cudaMemcpyHostToDevice,
                             e->own)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpyAsync(e->d_n_tiles, &n, sizeof(int), cudaMemcpyHostToDevice, e->own)) != cudaSuccess)
    return err;
  e->tiles_live = n_live;
  if ((err = cudaStreamSynchronize(e->own)) != cudaSuccess) return err;
  // one stream-collide block per `claim` tiles; the graphs hold the grid size
  const int grid = std::max(1, (n + e->claim - 1) / e->claim);
  if (grid != e->grid) {
    drop_graphs(e);
    e->grid = grid;
  }
  return cudaSuccess;
}

cudaError_t read_live(lbmd_ensemble *e, std::vector<int> &live) {
  live.assign(e->count, 0);
  cudaError_t err = cudaMemcpyAsync(live.data(), e->d_live + (e->G & 1) * e->count,
                                    e->count * sizeof(int), cudaMemcpyDeviceToHost, e->own);
  if (err != cudaSuccess) return err;
  return cudaStreamSynchronize(e->own);
}

cudaError_t read_status(lbmd_ensemble *e, std::vector<DevStatus> &st) {
  st.resize(e->count);
  cudaError_t err;
  for (int m = 0; m < e->count; ++m)
    if ((err = cudaMemcpyAsync(&st[m], e->inst[m].status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                               e->own)) != cudaSuccess)
      return err;
  return cudaStreamSynchronize(e->own);
}

// Re-derive the live flags of the next step from the status words and the
// cap (host side), move a resuming realisation's populations to the buffer
// the next step reads, and rebuild the tile list.
cudaError_t refresh_live(lbmd_ensemble *e) {
  std::vector<DevStatus> st;
  cudaError_t err;
  if ((err = read_status(e, st)) != cudaSuccess) return err;
  std::vector<int> live(e->count, 0);
  const int cur = (int)(e->G & 1);
  for (int m = 0; m < e->count; ++m) {
    live[m] = st[m].state == LBMD_RUNNING && st[m].step < e->cap;
    if (live[m] && st[m].out_buf != cur) {
      // its last output is in pop[out_buf]; the next step reads pop[cur]
      const size_t bytes = (size_t)19 * e->E.L[m].Vp * store_bytes(e->storage);
      if ((err = cudaMemcpyAsync(e->inst[m].pop[cur], e->inst[m].pop[st[m].out_buf], bytes,
                                 cudaMemcpyDeviceToDevice, e->own)) != cudaSuccess)
        return err;
    }
  }
  if ((err = cudaMemcpyAsync(e->d_live + cur * e->count, live.data(), e->count * sizeof(int),
                             cudaMemcpyHostToDevice, e->own)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpyAsync(e->d_cap, &e->cap, sizeof(long long), cudaMemcpyHostToDevice, e->own)) !=
      cudaSuccess)
    return err;
  return upload_tiles(e, live);  // synchronises: `live` and `cap` outlive the copies
}

// One ensemble step reading pop[cur] of every live realisation.  Without a
// solvent only the MD groups and the spread (bookkeeping: no transfer nodes)
// run.
cudaError_t enqueue_ens_step(lbmd_ensemble *e, int cur) {
  cudaError_t err;
  cudaEvent_t t[4] = {nullptr, nullptr, nullptr, nullptr};
  if (e->timing) {
    if (e->tev_used + 4 > e->tev.size())
      for (int k = 0; k < 400; ++k) {
        cudaEvent_t ev;
        if ((err = cudaEventCreate(&ev)) != cudaSuccess) return err;
        e->tev.push_back(ev);
      }
    for (int k = 0; k < 4; ++k) t[k] = e->tev[e->tev_used + k];
    e->tev_used += 4;
  }
  const int *live = e->d_live + cur * e->count;
  int *live_next = e->d_live + (cur ^ 1) * e->count;
  if (t[0] && (err = cudaEventRecord(t[0], e->own)) != cudaSuccess) return err;
  if (!e->solvent_free &&
      (err = launch_ens_gather(e->storage, e->d_mem, e->d_beads, e->E.nb, live, cur,
                               e->own)) != cudaSuccess)
    return err;
  if ((err = cudaEventRecord(e->ev_fork, e->own)) != cudaSuccess) return err;
  for (int s = 0; s < e->nside; ++s)
    if ((err = cudaStreamWaitEvent(e->side[s], e->ev_fork, 0)) != cudaSuccess) return err;
  for (size_t k = 0; k < e->groups.size(); ++k) {
    const Group &g = e->groups[k];
    if ((err = launch_ens_md_cycle(e->d_mem, e->d_chains + g.first, g.count, g.threads, g.max_n, live,
                                   e->prio_high, e->side[k % e->nside])) != cudaSuccess)
      return err;
  }
  if (t[1] && (err = cudaEventRecord(t[1], e->own)) != cudaSuccess) return err;
  if (!e->solvent_free &&
      (err = launch_ens_stream_collide(e->storage, e->forcing, e->rows, e->warps, e->cpt, e->claim, e->grid,
                                       e->d_lbd, e->d_tiles, e->d_n_tiles, live, cur,
                                       e->own)) != cudaSuccess)
    return err;
  if (t[2] && (err = cudaEventRecord(t[2], e->own)) != cudaSuccess) return err;
  if (!e->solvent_free) {
    // the sum part of the spread once every MD group is done, still beside
    // the stream-collide
    for (int s = 1; s < e->nside; ++s) {
      if ((err = cudaEventRecord(e->ev_join[s], e->side[s])) != cudaSuccess) return err;
      if ((err = cudaStreamWaitEvent(e->side[0], e->ev_join[s], 0)) != cudaSuccess) return err;
    }
    if ((err = launch_ens_spread_accum(e->d_mem, e->d_beads, e->E.nb, live, e->side[0])) !=
        cudaSuccess)
      return err;
  }
  for (int s = 0; s < e->nside; ++s) {
    if ((err = cudaEventRecord(e->ev_join[s], e->side[s])) != cudaSuccess) return err;
    if ((err = cudaStreamWaitEvent(e->own, e->ev_join[s], 0)) != cudaSuccess) return err;
  }
  if ((err = launch_ens_spread(e->storage, e->d_mem, e->d_beads, e->E.nb, live, live_next, cur,
                               e->d_cap, e->own)) != cudaSuccess)
    return err;
  if (t[3] && (err = cudaEventRecord(t[3], e->own)) != cudaSuccess) return err;
  return cudaSuccess;
}

cudaError_t capture_ens(lbmd_ensemble *e, int start, int nsteps, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamBeginCapture(e->own, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return err;
  cudaError_t err2 = cudaSuccess;
  int b = start;
  for (int k = 0; k < nsteps && err2 == cudaSuccess; ++k) {
    err2 = enqueue_ens_step(e, b);
    b ^= 1;
  }
  err = cudaStreamEndCapture(e->own, &g);
  if (err2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return err2;
  }
  if (err != cudaSuccess) return err;
  err = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  return err;
}

// Enqueue n steps on the private stream (graphs unless timing).
int enqueue_steps(lbmd_ensemble *e, int64_t n) {
  if (e->timing) {
    for (int64_t k = 0; k < n; ++k) {
      EK(e, enqueue_ens_step(e, (int)(e->G & 1)));
      e->G += 1;
    }
    return LBMD_OK;
  }
  int64_t left = n;
  for (int gi = 2; gi >= 0; --gi) {
    const int len = kEnsGraphSteps[gi];
    while (left >= len) {
      const int cur = (int)(e->G & 1);
      if (!e->graph[cur][gi]) EK(e, capture_ens(e, cur, len, &e->graph[cur][gi]));
      EK(e, cudaGraphLaunch(e->graph[cur][gi], e->own));
      e->G += len;
      left -= len;
    }
  }
  return LBMD_OK;
}

// One stream-collide block per `claim` tiles of the current tile list.  A
// new grid size drops the captured graphs (they hold the old one).
int set_grid(lbmd_ensemble *e) {
  const int per_sm = ens_lb_blocks_per_sm(e->storage, e->forcing, e->rows, e->warps, e->cpt);
  if (per_sm < 1) return fail(LBMD_EINVAL, "no ensemble stream-collide of this launch shape");
  const int grid = std::max(1, (int)((e->htiles.size() + e->claim - 1) / e->claim));
  if (grid != e->grid) drop_graphs(e);
  e->grid = grid;
  return LBMD_OK;
}

void destroy_ens(lbmd_ensemble *e) {
  if (!e) return;
  drop_graphs(e);
  for (cudaEvent_t ev : e->tev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {e->ev_in, e->ev_out, e->ev_fork})
    if (ev) cudaEventDestroy(ev);
  for (int s = 0; s < kEnsSide; ++s) {
    if (e->ev_join[s]) cudaEventDestroy(e->ev_join[s]);
    if (e->side[s]) cudaStreamDestroy(e->side[s]);
  }
  if (e->own) cudaStreamDestroy(e->own);
  delete e;
}

}  // namespace

extern "C" {

int lbmd_ensemble_workspace_size(const lbmd_params *members, int32_t count, size_t *bytes) {
  int rc = validate_members(members, count);
  if (rc) return rc;
  if (!bytes) return fail(LBMD_EINVAL, "bytes is NULL");
  *bytes = make_ens_layout(members, count).total;
  return LBMD_OK;
}

int lbmd_ensemble_create(const lbmd_params *members, int32_t count, void *dev_workspace,
                         size_t bytes, void *cuda_stream, lbmd_ensemble **out) {
  if (!out) return fail(LBMD_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate_members(members, count);
  if (rc) return rc;
  // members without init_pos start from the library's seeded walk
  std::vector<lbmd_params> given(members, members + count);
  std::vector<std::vector<double>> starts(count);
  for (int m = 0; m < count; ++m)
    if (!given[m].init_pos) {
      if ((rc = seeded_start(given[m], starts[m])) != LBMD_OK) {
        char buf[512];
        snprintf(buf, sizeof(buf), "%s", last_message());
        return fail(rc, "member %d: %s", m, buf);
      }
      given[m].init_pos = starts[m].data();
    }
  members = given.data();
  EnsLayout E = make_ens_layout(members, count);
  if (!dev_workspace || bytes < E.total)
    return fail(LBMD_ESIZE, "workspace of %zu bytes, %zu needed", bytes, E.total);
  if (((uintptr_t)dev_workspace) % kAlign)
    return fail(LBMD_ESIZE, "workspace must be %zu-byte aligned", kAlign);

  lbmd_ensemble *e = new (std::nothrow) lbmd_ensemble();
  if (!e) return fail(LBMD_EINVAL, "host allocation failed");
  e->count = count;
  e->storage = members[0].storage;
  e->forcing = members[0].forcing;
  e->solvent_free = members[0].solvent_free;
  {
    bool no_force = true;
    for (int m = 0; m < count; ++m)
      for (int a = 0; a < 3; ++a) no_force = no_force && members[m].body_force[a] == 0.0;
    if (no_force) e->forcing = kForcingNone;  // collision variant of the stream-collide
  }
  e->p.assign(members, members + count);
  for (auto &q : e->p) {
    q.bond_i = q.bond_j = nullptr;
    q.bond_len = q.init_pos = q.init_vel = q.init_rho = q.init_u = nullptr;
  }
  e->E = E;
  e->ws = (char *)dev_workspace;
  e->user = (cudaStream_t)cuda_stream;
  e->d_mem = (EnsMember *)(e->ws + E.mem);
  e->d_lbd = (EnsLb *)(e->ws + E.lbd);
  e->d_tiles = (EnsTile *)(e->ws + E.tiles);
  e->d_n_tiles = (int *)(e->ws + E.n_tiles);
  e->d_beads = (int2 *)(e->ws + E.beads);
  e->d_live = (int *)(e->ws + E.live);
  e->d_cap = (long long *)(e->ws + E.cap);
  e->d_chains = (int *)(e->ws + E.chains);
  e->stage = (float *)(e->ws + E.stage);
  e->rows = 8;
  e->warps = 48;
  e->claim = 2;
  e->cpt = 1;
  e->cap = LLONG_MAX;

  auto bail = [&](cudaError_t err, const char *what) {
    int r = ens_fail(nullptr, err, what);
    destroy_ens(e);
    return r;
  };
  cudaError_t err;
  int dev = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return bail(err, "device");
  if ((err = cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return bail(err, "SM count");
  if ((err = cudaStreamCreateWithFlags(&e->own, cudaStreamNonBlocking)) != cudaSuccess) return bail(err, "stream");
  int prio_least = 0;
  if ((err = cudaDeviceGetStreamPriorityRange(&prio_least, &e->prio_high)) != cudaSuccess)
    return bail(err, "priority range");
  for (int s = 0; s < kEnsSide; ++s) {
    if ((err = cudaStreamCreateWithPriority(&e->side[s], cudaStreamNonBlocking, e->prio_high)) != cudaSuccess)
      return bail(err, "stream");
    if ((err = cudaEventCreateWithFlags(&e->ev_join[s], cudaEventDisableTiming)) != cudaSuccess)
      return bail(err, "event");
  }
  for (cudaEvent_t *ev : {&e->ev_in, &e->ev_out, &e->ev_fork})
    if ((err = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return bail(err, "event");

  // every realisation as a single box in its slice (synchronises per member)
  e->inst.resize(count);
  e->hmem.resize(count);
  e->hlbd.resize(count);
  for (int m = 0; m < count; ++m) {
    const char *what = "create";
    if ((err = init_instance(members[m], E.L[m], e->ws + E.off[m], e->user, e->inst[m], &what)) !=
        cudaSuccess)
      return bail(err, what);
    EnsMember &M = e->hmem[m];
    memset(&M, 0, sizeof(M));
    M.a = e->inst[m].chain;
    M.a.f = nullptr;
    M.a.f_mode = kPopPull;
    M.ph = e->inst[m].phys;
    M.pop[0] = e->inst[m].pop[0];
    M.pop[1] = e->inst[m].pop[1];
    EnsLb &D = e->hlbd[m];
    memset(&D, 0, sizeof(D));
    const LbGeom &g = e->inst[m].geo;
    D.pop[0] = M.pop[0];
    D.pop[1] = M.pop[1];
    D.lmask = g.lmask;
    D.tile_near = g.tile_near;
    D.nx = g.nx;
    D.ny = g.ny;
    D.nz = g.nz;
    D.ntx = g.ntx;
    D.Vp = (int)g.Vp;
    D.inv_nx = 1.0f / (float)g.nx;
    D.omega = M.ph.omega;
    D.rho0 = M.ph.rho0;
    for (int a = 0; a < 3; ++a) D.g[a] = M.ph.g[a];
    D.forcing = M.ph.forcing;
    D.nonfinite = M.ph.nonfinite;
  }
  // (realisation, bead) slots, each realisation padded to a multiple of four
  std::vector<int2> beads;
  beads.reserve(E.nb);
  for (int m = 0; m < count; ++m) {
    const int N = members[m].n_beads, Np = (N + 3) / 4 * 4;
    for (int i = 0; i < Np; ++i) beads.push_back(i < N ? make_int2(m, i) : make_int2(-1, 0));
  }
  // MD groups: chains with the same block size (one thread per bead, whole warps)
  std::map<int, std::vector<int>> by_threads;
  for (int m = 0; m < count; ++m) by_threads[md_threads(members[m].n_beads)].push_back(m);
  std::vector<int> chains;
  for (auto &kv : by_threads) {
    Group g{kv.first, 0, (int)chains.size(), (int)kv.second.size()};
    for (int m : kv.second) {
      chains.push_back(m);
      g.max_n = std::max(g.max_n, members[m].n_beads);
    }
    e->groups.push_back(g);
  }
  e->nside = std::min<int>(kEnsSide, std::max<int>(1, (int)e->groups.size()));
  std::vector<int> live0(2 * (size_t)count, 0);
  std::fill(live0.begin(), live0.begin() + count, 1);
  cudaStream_t s = e->user;
  if ((err = cudaMemcpyAsync(e->d_mem, e->hmem.data(), count * sizeof(EnsMember), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaMemcpyAsync(e->d_lbd, e->hlbd.data(), count * sizeof(EnsLb), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaMemcpyAsync(e->d_beads, beads.data(), beads.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaMemcpyAsync(e->d_chains, chains.data(), chains.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaMemcpyAsync(e->d_live, live0.data(), live0.size() * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaMemcpyAsync(e->d_cap, &e->cap, sizeof(long long), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(err, "upload");
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return bail(err, "create sync");
  if ((rc = set_grid(e))) {
    destroy_ens(e);
    return rc;
  }
  std::vector<int> all(count, 1);
  if ((err = upload_tiles(e, all)) != cudaSuccess) return bail(err, "tiles");
  *out = e;
  return LBMD_OK;
}

int lbmd_ensemble_step(lbmd_ensemble *e, int64_t n_steps) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (n_steps < 0) return fail(LBMD_EINVAL, "n_steps < 0");
  if (n_steps == 0) return LBMD_OK;
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  if ((rc = enqueue_steps(e, n_steps))) return rc;
  EK(e, cudaEventRecord(e->ev_out, e->own));
  EK(e, cudaStreamWaitEvent(e->user, e->ev_out, 0));
  return LBMD_OK;
}

int lbmd_ensemble_run(lbmd_ensemble *e, int64_t max_steps, int64_t check_every, int64_t *steps_run) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (max_steps < 0) return fail(LBMD_EINVAL, "max_steps < 0");
  if (check_every <= 0) check_every = 1024;
  check_every = (check_every + kEnsBlock - 1) / kEnsBlock * kEnsBlock;
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  e->cap = max_steps;
  EK(e, refresh_live(e));
  const long long G0 = e->G;
  std::vector<int> live;
  EK(e, read_live(e, live));
  int n_live = (int)std::count(live.begin(), live.end(), 1);
  while (n_live > 0) {
    if ((rc = enqueue_steps(e, check_every))) return rc;
    EK(e, read_live(e, live));
    n_live = (int)std::count(live.begin(), live.end(), 1);
    // drop finished realisations from the tile list once a quarter of the
    // listed ones are done
    if (n_live > 0 && 4 * (e->tiles_live - n_live) >= e->tiles_live) EK(e, upload_tiles(e, live));
  }
  if (steps_run) *steps_run = e->G - G0;
  EK(e, cudaEventRecord(e->ev_out, e->own));
  EK(e, cudaStreamWaitEvent(e->user, e->ev_out, 0));
  return LBMD_OK;
}

int lbmd_ensemble_results(lbmd_ensemble *e, int32_t *state, int64_t *t_transloc, int64_t *steps,
                          int32_t *n_trans) {
  int rc = check_ens(e);
  if (rc) return rc;
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  std::vector<DevStatus> st;
  EK(e, read_status(e, st));
  for (int m = 0; m < e->count; ++m) {
    if (state) state[m] = st[m].state;
    if (t_transloc) t_transloc[m] = st[m].t_transloc;
    if (steps) steps[m] = st[m].step;
    if (n_trans) n_trans[m] = st[m].n_trans;
  }
  return LBMD_OK;
}

int lbmd_ensemble_live(lbmd_ensemble *e, int32_t *n_live) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (!n_live) return fail(LBMD_EINVAL, "n_live is NULL");
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  std::vector<int> live;
  EK(e, read_live(e, live));
  *n_live = (int32_t)std::count(live.begin(), live.end(), 1);
  return LBMD_OK;
}

int lbmd_ensemble_read_beads(lbmd_ensemble *e, int32_t member, double *pos, double *vel,
                             int dst_is_device) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (member < 0 || member >= e->count) return fail(LBMD_EINVAL, "member out of range");
  const ChainArgs &a = e->inst[member].chain;
  const int N = a.N;
  if (!pos && !vel) return LBMD_OK;
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  double *dx = pos, *dy = vel;
  if (!dst_is_device) {
    dx = pos ? (double *)e->stage : nullptr;
    dy = vel ? (double *)e->stage + 3 * N : nullptr;
  }
  EK(e, launch_read_beads(a.pos, a.pos_lo, a.vel, N, a.ox, a.oy, a.oz, dx, dy, e->own));
  if (!dst_is_device) {
    if (pos) EK(e, cudaMemcpyAsync(pos, dx, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, e->own));
    if (vel) EK(e, cudaMemcpyAsync(vel, dy, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, e->own));
  }
  EK(e, cudaStreamSynchronize(e->own));
  return LBMD_OK;
}

int lbmd_ensemble_read_populations(lbmd_ensemble *e, int32_t member, float *f, int dst_is_device) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (member < 0 || member >= e->count) return fail(LBMD_EINVAL, "member out of range");
  if (!f) return fail(LBMD_EINVAL, "f is NULL");
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  DevStatus st;
  EK(e, cudaMemcpyAsync(&st, e->inst[member].status, sizeof(st), cudaMemcpyDeviceToHost, e->own));
  EK(e, cudaStreamSynchronize(e->own));
  const Instance &in = e->inst[member];
  const LbGeom &g = in.geo;
  const float rho0 = (float)e->p[member].rho0;
  const void *src = in.pop[st.out_buf & 1];
  if (dst_is_device) {
    EK(e, launch_read_pulled(e->storage, g, rho0, src, kPopPull, 0, g.nz, f, g.V, e->own));
    EK(e, cudaStreamSynchronize(e->own));
    return LBMD_OK;
  }
  const long long plane = (long long)g.nx * g.ny;
  const long long nzc_max = std::max(1LL, e->E.L[member].chunk_cells / plane);
  for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
    const long long nzc = std::min(nzc_max, (long long)g.nz - z0);
    const long long cells = nzc * plane;
    EK(e, launch_read_pulled(e->storage, g, rho0, src, kPopPull, z0, nzc, e->stage, cells, e->own));
    for (int q = 0; q < 19; ++q)
      EK(e, cudaMemcpyAsync(f + q * g.V + z0 * plane, e->stage + q * cells, cells * 4,
                            cudaMemcpyDeviceToHost, e->own));
  }
  EK(e, cudaStreamSynchronize(e->own));
  return LBMD_OK;
}

int lbmd_ensemble_read_diagnostics(lbmd_ensemble *e, int32_t member, lbmd_diag *records,
                                   int32_t max_records, int32_t *n_records) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (member < 0 || member >= e->count) return fail(LBMD_EINVAL, "member out of range");
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  const Instance &in = e->inst[member];
  return copy_diagnostics(in.status, in.chain.diag, e->p[member].diag_capacity, records,
                          max_records, n_records, e->own);
}

int lbmd_ensemble_set_tuning(lbmd_ensemble *e, int32_t rows, int32_t warps, int32_t claim,
                             int32_t cells_per_thread) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (rows != 4 && rows != 8 && rows != 16) return fail(LBMD_EINVAL, "rows must be 4, 8 or 16");
  if (warps != 32 && warps != 48) return fail(LBMD_EINVAL, "warps must be 32 or 48");
  if (claim < 1 || claim > 64) return fail(LBMD_EINVAL, "claim must be in [1, 64]");
  if (cells_per_thread != 1 && cells_per_thread != 2 && cells_per_thread != kEnsXPair)
    return fail(LBMD_EINVAL, "cells_per_thread must be 1, 2 or LBMD_ENS_XPAIR");
  if (cells_per_thread != 1 && (warps != 32 || rows == 16))
    return fail(LBMD_EINVAL, "two cells per thread need warps = 32 and rows 4 or 8");
  if (cells_per_thread == kEnsXPair && !xpair_ok(e))
    return fail(LBMD_EINVAL, "x-adjacent pairs need 16-bit storage and an even nx in every member");
  EK(e, cudaStreamSynchronize(e->own));
  const bool retile = rows != e->rows || cells_per_thread != e->cpt;
  e->rows = rows;
  e->warps = warps;
  e->claim = claim;
  e->cpt = cells_per_thread;
  if ((rc = set_grid(e))) return rc;
  drop_graphs(e);
  if (retile) {
    std::vector<int> live;
    EK(e, read_live(e, live));
    EK(e, upload_tiles(e, live));
  }
  return LBMD_OK;
}

int lbmd_ensemble_get_tuning(lbmd_ensemble *e, int32_t *rows, int32_t *warps, int32_t *claim,
                             int32_t *cells_per_thread) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (rows) *rows = e->rows;
  if (warps) *warps = e->warps;
  if (claim) *claim = e->claim;
  if (cells_per_thread) *cells_per_thread = e->cpt;
  return LBMD_OK;
}

int lbmd_ensemble_autotune(lbmd_ensemble *e, int32_t trials, double *best_ms) {
  int rc = check_ens(e);
  if (rc) return rc;
  if (trials < 1) return fail(LBMD_EINVAL, "trials must be >= 1");
  if (e->solvent_free) {  // no stream-collide to tune
    if (best_ms) *best_ms = 0.0;
    return LBMD_OK;
  }
  EK(e, cudaEventRecord(e->ev_in, e->user));
  EK(e, cudaStreamWaitEvent(e->own, e->ev_in, 0));
  cudaEvent_t t0, t1;
  EK(e, cudaEventCreate(&t0));
  if (cudaEventCreate(&t1) != cudaSuccess) {
    cudaEventDestroy(t0);
    return fail(LBMD_ECUDA, "event");
  }
  const int cur = (int)(e->G & 1);
  const int *live = e->d_live + cur * e->count;
  double best = 1e30;
  int br = e->rows, bw = e->warps, bc = e->claim, bz = e->cpt;
  cudaError_t err = cudaSuccess;
  std::vector<int> hl;
  if ((err = read_live(e, hl)) != cudaSuccess) goto done;
  for (int cpt : {1, 2, kEnsXPair})
  for (int rows : {4, 8, 16}) {
    if (cpt == kEnsXPair && !xpair_ok(e)) continue;
    e->rows = rows;
    e->cpt = cpt;
    if ((err = upload_tiles(e, hl)) != cudaSuccess) goto done;
    for (int warps : {32, 48}) {
      const int per_sm = ens_lb_blocks_per_sm(e->storage, e->forcing, rows, warps, cpt);
      if (per_sm < 1) continue;
      for (int claim : {1, 2, 4, 8}) {
        // one untimed launch, then `trials` timed ones
        const int grid = std::max(1, (int)((e->htiles.size() + claim - 1) / claim));
        for (int k = 0; k <= trials; ++k) {
          if (k == 1 && (err = cudaEventRecord(t0, e->own)) != cudaSuccess) goto done;
          if ((err = launch_ens_stream_collide(e->storage, e->forcing, rows, warps, cpt, claim, grid,
                                               e->d_lbd, e->d_tiles, e->d_n_tiles, live, cur,
                                               e->own)) != cudaSuccess)
            goto done;
        }
        if ((err = cudaEventRecord(t1, e->own)) != cudaSuccess) goto done;
        if ((err = cudaEventSynchronize(t1)) != cudaSuccess) goto done;
        float ms = 0.f;
        if ((err = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) goto done;
        const double avg = ms / trials;
        if (avg < best) {
          best = avg;
          br = rows;
          bw = warps;
          bc = claim;
          bz = cpt;
        }
      }
    }
  }
done:
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (err != cudaSuccess) return ens_fail(e, err, "autotune");
  e->rows = br;
  e->warps = bw;
  e->claim = bc;
  e->cpt = bz;
  if ((rc = set_grid(e))) return rc;
  drop_graphs(e);
  EK(e, upload_tiles(e, hl));
  EK(e, cudaEventRecord(e->ev_out, e->own));
  EK(e, cudaStreamWaitEvent(e->user, e->ev_out, 0));
  if (best_ms) *best_ms = best;
  return LBMD_OK;
}

int lbmd_ensemble_set_kernel_timing(lbmd_ensemble *e, int enable) {
  int rc = check_ens(e);
  if (rc) return rc;
  EK(e, cudaStreamSynchronize(e->own));
  e->timing = enable ? 1 : 0;
  e->tev_used = 0;
  e->timed_lb = e->timed_step = 0;
  e->timed_count = 0;
  return LBMD_OK;
}

int lbmd_ensemble_kernel_times(lbmd_ensemble *e, double *lb_ms, double *step_ms, int64_t *steps) {
  int rc = check_ens(e);
  if (rc) return rc;
  EK(e, cudaStreamSynchronize(e->own));
  for (int s = 0; s < e->nside; ++s) EK(e, cudaStreamSynchronize(e->side[s]));
  for (size_t k = 0; k + 3 < e->tev_used; k += 4) {
    float a = 0.f, b = 0.f;
    EK(e, cudaEventElapsedTime(&a, e->tev[k + 1], e->tev[k + 2]));
    EK(e, cudaEventElapsedTime(&b, e->tev[k], e->tev[k + 3]));
    e->timed_lb += a;
    e->timed_step += b;
    e->timed_count += 1;
  }
  e->tev_used = 0;
  if (lb_ms) *lb_ms = e->timed_lb;
  if (step_ms) *step_ms = e->timed_step;
  if (steps) *steps = e->timed_count;
  return LBMD_OK;
}

int lbmd_ensemble_destroy(lbmd_ensemble *e) {
  if (!e) return LBMD_OK;
  cudaStreamSynchronize(e->own);
  for (int s = 0; s < kEnsSide; ++s)
    if (e->side[s]) cudaStreamSynchronize(e->side[s]);
  destroy_ens(e);
  return LBMD_OK;
}

}  // extern "C"
