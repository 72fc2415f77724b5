// lbmd_abi.cu -- the C ABI of include/lbmd.h: parameter checks, the Sec. III
// geometry, the workspace layout, CUDA-graph capture of the coupled step and
// the read-outs.  No device memory is allocated here: every buffer is carved
// out of the caller's workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lbmd_internal.h"

using namespace lbmd;

namespace {

thread_local char g_msg[512] = "";

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t store_bytes(int storage) { return storage == LBMD_STORE_F32 ? 4 : 2; }

struct Layout {
  size_t popA, popB, solid, tile, xslab, pos, pos_lo, vel, ui, J, sp_node, sp_w, b0, nl_cnt, wl_cnt,
      nl_list, wl_list, nl_ref, lam, status, stage;
  size_t stage_floats;  // staging capacity in floats
  size_t total;
  long long Vp;
  int ntx;
  long long chunk_cells;
};

Layout make_layout(const lbmd_params &p) {
  Layout L{};
  const long long V = (long long)p.nx * p.ny * p.nz;
  L.Vp = (V + 63) / 64 * 64;
  L.ntx = (p.nx + 31) / 32;
  const size_t rows = (size_t)p.ny * p.nz;
  const size_t Np = (size_t)std::max(p.n_beads, 1);
  const long long plane = (long long)p.nx * p.ny;
  L.chunk_cells = std::min(V, std::max(plane, (long long)(1 << 20)));
  L.chunk_cells = (L.chunk_cells / plane) * plane;  // whole z-planes
  if (L.chunk_cells < plane) L.chunk_cells = plane;
  L.stage_floats = std::max((size_t)19 * (size_t)L.chunk_cells, (size_t)6 * Np * 2);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.popA = take((size_t)19 * L.Vp * store_bytes(p.storage));
  L.popB = take((size_t)19 * L.Vp * store_bytes(p.storage));
  L.solid = take(rows * L.ntx * sizeof(uint32_t));
  L.tile = take(rows * L.ntx);
  L.xslab = take((size_t)p.nx);
  L.pos = take(Np * sizeof(float4));
  L.pos_lo = take(Np * sizeof(float4));
  L.vel = take(Np * sizeof(float4));
  L.ui = take(Np * sizeof(float4));
  L.J = take(Np * sizeof(float4));
  L.sp_node = take(8 * Np * sizeof(int));
  L.sp_w = take(8 * Np * sizeof(float));
  L.b0 = take(Np * sizeof(double));
  L.nl_cnt = take(Np * sizeof(int));
  L.wl_cnt = take(Np * sizeof(int));
  L.nl_list = take(Np * kMaxPairs * sizeof(short));
  L.wl_list = take(Np * kMaxWall * sizeof(float4));
  L.nl_ref = take(Np * sizeof(float4));
  L.lam = take(Np * sizeof(float));
  L.status = take(sizeof(DevStatus));
  L.stage = take(L.stage_floats * sizeof(float));
  L.total = o;
  return L;
}

int validate(const lbmd_params *p) {
  if (!p) return fail(LBMD_EINVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBMD_EINVAL, "box dimensions must be >= 1");
  const long long V = (long long)p->nx * p->ny * p->nz;
  if (V > 0x7fffffffLL) return fail(LBMD_EINVAL, "box has more than 2^31-1 nodes");
  if (p->nz > 65535) return fail(LBMD_EINVAL, "nz must be <= 65535");
  if (p->storage < LBMD_STORE_F32 || p->storage > LBMD_STORE_BF16)
    return fail(LBMD_EINVAL, "unknown storage %d", p->storage);
  if (p->forcing != LBMD_FORCING_PAPER && p->forcing != LBMD_FORCING_GUO)
    return fail(LBMD_EINVAL, "unknown forcing %d", p->forcing);
  if (p->coupling != LBMD_COUPLING_TRILINEAR && p->coupling != LBMD_COUPLING_NGP)
    return fail(LBMD_EINVAL, "unknown coupling %d", p->coupling);
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBMD_EINVAL, "tau must be > 1/2");
  if (!(p->rho0 > 0)) return fail(LBMD_EINVAL, "rho0 must be > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->body_force[a])) return fail(LBMD_EINVAL, "body force not finite");
  if (p->wall_x < -1 || p->wall_x >= p->nx) return fail(LBMD_EINVAL, "wall_x out of range");
  if (p->wall_x >= 0) {
    if (p->wall_thickness < 1 || p->wall_thickness >= p->nx)
      return fail(LBMD_EINVAL, "wall_thickness must be in [1, nx)");
    if (p->pore_d < 0 || p->pore_d > p->ny || p->pore_d > p->nz)
      return fail(LBMD_EINVAL, "pore_d out of range");
    if (p->pore_y0 < -1 || p->pore_z0 < -1 || p->pore_y0 + p->pore_d > p->ny ||
        p->pore_z0 + p->pore_d > p->nz)
      return fail(LBMD_EINVAL, "pore origin out of range");
  }
  if (p->y_walls != 0 && p->y_walls != 1) return fail(LBMD_EINVAL, "y_walls must be 0 or 1");
  if (p->y_walls && p->ny < 3) return fail(LBMD_EINVAL, "y_walls needs ny >= 3");
  if (p->n_beads < 0 || p->n_beads > LBMD_MAX_BEADS)
    return fail(LBMD_EINVAL, "n_beads must be in [0, %d]", LBMD_MAX_BEADS);
  if (p->n_beads > 0) {
    if (p->md_substeps < 1 || p->md_substeps > 255)
      return fail(LBMD_EINVAL, "md_substeps must be in [1, 255]");
    if (!p->init_pos) return fail(LBMD_EINVAL, "init_pos is required when n_beads > 0");
    if (!(p->bead_mass > 0) || !(p->gamma >= 0) || !(p->kT >= 0) || !(p->lj_sigma > 0) ||
        !(p->lj_eps >= 0) || !(p->kappa_phi >= 0) || !std::isfinite(p->f_drive))
      return fail(LBMD_EINVAL, "bead parameters out of range");
    if (p->n_constraints < -1) return fail(LBMD_EINVAL, "n_constraints must be >= -1");
    if (p->n_constraints == -1 && p->n_beads > 1 && !(p->bond_length > 0))
      return fail(LBMD_EINVAL, "bond_length must be > 0");
    if (p->n_constraints > 0) {
      if (!p->bond_i || !p->bond_j || !p->bond_len)
        return fail(LBMD_EINVAL, "bond arrays are required when n_constraints > 0");
      if (p->n_constraints != p->n_beads - 1)
        return fail(LBMD_EUNSUPPORTED, "only a linear chain of n_beads-1 bonds is supported");
      for (int k = 0; k < p->n_constraints; ++k) {
        if (p->bond_i[k] != k || p->bond_j[k] != k + 1)
          return fail(LBMD_EUNSUPPORTED, "bond %d is not (k, k+1): only linear chains", k);
        if (!(p->bond_len[k] > 0)) return fail(LBMD_EINVAL, "bond %d length must be > 0", k);
      }
    }
    const bool bonds = p->n_constraints == -1 ? p->n_beads > 1 : p->n_constraints > 0;
    if (bonds && (p->shake_max_iter < 1 || !(p->shake_tol > 0)))
      return fail(LBMD_EINVAL, "shake_max_iter >= 1 and shake_tol > 0 required");
    for (int i = 0; i < 3 * p->n_beads; ++i)
      if (!std::isfinite(p->init_pos[i])) return fail(LBMD_EINVAL, "init_pos not finite");
  }
  return LBMD_OK;
}

void pore_origin(const lbmd_params &p, int &y0, int &z0) {
  y0 = p.pore_y0 >= 0 ? p.pore_y0 : (p.ny - p.pore_d) / 2;
  z0 = p.pore_z0 >= 0 ? p.pore_z0 : (p.nz - p.pore_d) / 2;
}

// Solid nodes of Sec. III: the wall layers minus the centred pore, plus the
// optional rows y = 0 and y = ny - 1.
bool is_solid(const lbmd_params &p, int x, int y, int z) {
  if (p.y_walls && (y == 0 || y == p.ny - 1)) return true;
  if (p.wall_x < 0) return false;
  bool in_wall = false;
  for (int t = 0; t < p.wall_thickness; ++t)
    if (x == (p.wall_x + t) % p.nx) in_wall = true;
  if (!in_wall) return false;
  int y0, z0;
  pore_origin(p, y0, z0);
  const bool in_pore = p.pore_d > 0 && y >= y0 && y < y0 + p.pore_d && z >= z0 && z < z0 + p.pore_d;
  return !in_pore;
}

struct HostGeometry {
  std::vector<uint32_t> bits;   // [nz][ny][ntx]
  std::vector<uint8_t> tile;    // [nz][ny][ntx]
  std::vector<uint8_t> xslab;   // [nx]
};

void build_geometry(const lbmd_params &p, int ntx, HostGeometry &G) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  G.bits.assign((size_t)nz * ny * ntx, 0u);
  G.tile.assign((size_t)nz * ny * ntx, 0u);
  G.xslab.assign((size_t)nx, 0u);
  const bool any_solid = p.y_walls || p.wall_x >= 0;
  if (!any_solid) return;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        if (is_solid(p, x, y, z)) {
          G.bits[((size_t)z * ny + y) * ntx + (x >> 5)] |= 1u << (x & 31);
          G.xslab[x] = 1;
        }
  std::vector<uint8_t> col((size_t)nx);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      // solid anywhere in the 3x3 rows around (y, z), per x
      std::fill(col.begin(), col.end(), 0);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
          const int yy = ((y + dy) % ny + ny) % ny, zz = ((z + dz) % nz + nz) % nz;
          for (int w = 0; w < ntx; ++w) {
            const uint32_t word = G.bits[((size_t)zz * ny + yy) * ntx + w];
            if (!word) continue;
            for (int b = 0; b < 32; ++b)
              if ((word >> b) & 1u) col[(size_t)w * 32 + b] = 1;
          }
        }
      for (int t = 0; t < ntx; ++t) {
        const int x0 = t * 32, x1 = std::min(nx - 1, x0 + 31);
        uint8_t near = 0;
        for (int x = x0 - 1; x <= x1 + 1 && !near; ++x) near |= col[(size_t)((x % nx) + nx) % nx];
        G.tile[((size_t)z * ny + y) * ntx + t] = near;
      }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
struct lbmd_ctx {
  lbmd_params p;  // host pointers cleared after create
  Layout L;
  LbGeom geo;
  LbPhys phys;
  ChainArgs chain;
  char *ws;
  char *pop[2];
  int cur;  // pop[cur] holds the post-collision populations of the last step
  int N, has_bonds;
  cudaStream_t user;        // caller's stream
  cudaStream_t own, side;   // private streams: steps run on own, MD on side
  int prio_high;            // greatest stream priority of the device
  cudaEvent_t ev_in, ev_out, ev_fork, ev_join;
  cudaGraphExec_t graph[2][3];  // [starting buffer][1, 2, kBlockSteps steps]
  int sticky;
  int timing;
  std::vector<cudaEvent_t> tev;  // per timed step: lb, md, spread start/stop pairs
  size_t tev_used;
  double timed_ms[3];            // summed durations of stream-collide, MD, spread
  long long timed_count;
  DevStatus *status;
  float *stage;
};

namespace {

constexpr int kBlockSteps = 16;
const int kGraphSteps[3] = {1, 2, kBlockSteps};

int cuda_fail(lbmd_ctx *c, cudaError_t e, const char *what) {
  if (c) c->sticky = LBMD_ECUDA;
  return fail(LBMD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
#define CK(ctx, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Enqueue one coupled LB step reading pop[src] and writing pop[1 - src] on
// the private stream `own`: the MD cycle (gather + M substeps) on the side
// stream concurrently with the stream-collide, then the spread of the bead
// impulses into the new post-collision populations.  With paper forcing the
// bead source does not depend on f, so adding it after the collision is exact.
cudaError_t enqueue_step(lbmd_ctx *c, int src) {
  const void *A = c->pop[src];
  void *B = c->pop[1 - src];
  cudaError_t e;
  cudaEvent_t t[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (c->timing) {
    if (c->tev_used + 6 > c->tev.size()) {
      for (int k = 0; k < 600; ++k) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        c->tev.push_back(ev);
      }
    }
    for (int k = 0; k < 6; ++k) t[k] = c->tev[c->tev_used + k];
    c->tev_used += 6;
  }
  if (c->N > 0) {
    // (1) gather from the pre-step populations, then fork: the MD cycle runs
    // on the side stream while the stream-collide runs on the main one
    ChainArgs a = c->chain;
    a.f = A;
    if (t[2] && (e = cudaEventRecord(t[2], c->own)) != cudaSuccess) return e;
    if ((e = launch_gather(c->p.storage, a, c->own)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->ev_fork, c->own)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->side, c->ev_fork, 0)) != cudaSuccess) return e;
    if ((e = launch_md_cycle(a, c->prio_high, c->side)) != cudaSuccess) return e;
    if (t[3] && (e = cudaEventRecord(t[3], c->side)) != cudaSuccess) return e;
  } else if (t[2]) {
    if ((e = cudaEventRecord(t[2], c->own)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t[3], c->own)) != cudaSuccess) return e;
  }
  if (t[0] && (e = cudaEventRecord(t[0], c->own)) != cudaSuccess) return e;
  if ((e = launch_lb_stream_collide(c->p.storage, c->geo, c->phys, A, B,
                                    c->N > 0 ? nullptr : c->status, c->own)) != cudaSuccess)
    return e;
  if (t[1] && (e = cudaEventRecord(t[1], c->own)) != cudaSuccess) return e;
  if (c->N > 0) {
    if ((e = cudaEventRecord(c->ev_join, c->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->own, c->ev_join, 0)) != cudaSuccess) return e;
    if (t[4] && (e = cudaEventRecord(t[4], c->own)) != cudaSuccess) return e;
    if ((e = launch_spread(c->p.storage, c->geo, c->chain.sp_node, c->chain.sp_w, c->chain.J, c->N,
                           8 * c->N, B, c->status, c->own)) != cudaSuccess)
      return e;
    if (t[5] && (e = cudaEventRecord(t[5], c->own)) != cudaSuccess) return e;
  } else if (t[4]) {
    if ((e = cudaEventRecord(t[4], c->own)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t[5], c->own)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t capture(lbmd_ctx *c, int start, int nsteps, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->own, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = cudaSuccess;
  int b = start;
  for (int k = 0; k < nsteps && e2 == cudaSuccess; ++k) {
    e2 = enqueue_step(c, b);
    b ^= 1;
  }
  e = cudaStreamEndCapture(c->own, &g);
  if (e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e2;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  return e;
}

void destroy_ctx(lbmd_ctx *c) {
  if (!c) return;
  for (auto &row : c->graph)
    for (auto &gx : row)
      if (gx) cudaGraphExecDestroy(gx);
  for (cudaEvent_t ev : c->tev) cudaEventDestroy(ev);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->own) cudaStreamDestroy(c->own);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

int check_ctx(lbmd_ctx *c) {
  if (!c) return fail(LBMD_EINVAL, "context is NULL");
  if (c->sticky) return c->sticky;
  return LBMD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int lbmd_version(void) { return (1 << 16) | 0; }

const char *lbmd_last_message(void) { return g_msg; }

const char *lbmd_strerror(int status) {
  switch (status) {
    case LBMD_OK: return "ok";
    case LBMD_EINVAL: return "invalid argument";
    case LBMD_ESIZE: return "workspace too small or misaligned";
    case LBMD_ECUDA: return "CUDA error";
    case LBMD_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

int lbmd_workspace_size(const lbmd_params *params, size_t *bytes) {
  int rc = validate(params);
  if (rc) return rc;
  if (!bytes) return fail(LBMD_EINVAL, "bytes is NULL");
  *bytes = make_layout(*params).total;
  return LBMD_OK;
}

int lbmd_create(const lbmd_params *params, void *dev_workspace, size_t bytes, void *cuda_stream,
                lbmd_ctx **out) {
  if (!out) return fail(LBMD_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  const lbmd_params &p = *params;
  Layout L = make_layout(p);
  if (!dev_workspace || bytes < L.total)
    return fail(LBMD_ESIZE, "workspace of %zu bytes, %zu needed", bytes, L.total);
  if (((uintptr_t)dev_workspace) % kAlign)
    return fail(LBMD_ESIZE, "workspace must be %zu-byte aligned", kAlign);

  lbmd_ctx *c = new (std::nothrow) lbmd_ctx();
  if (!c) return fail(LBMD_EINVAL, "host allocation failed");
  c->p = p;
  c->p.bond_i = c->p.bond_j = nullptr;
  c->p.bond_len = c->p.init_pos = c->p.init_vel = c->p.init_rho = c->p.init_u = nullptr;
  c->L = L;
  c->ws = (char *)dev_workspace;
  c->pop[0] = c->ws + L.popA;
  c->pop[1] = c->ws + L.popB;
  c->cur = 0;
  c->user = (cudaStream_t)cuda_stream;
  c->N = p.n_beads;
  c->has_bonds = (p.n_constraints == -1 ? p.n_beads > 1 : p.n_constraints > 0) ? 1 : 0;
  c->status = (DevStatus *)(c->ws + L.status);
  c->stage = (float *)(c->ws + L.stage);

  auto bail = [&](cudaError_t e, const char *what) {
    int r = cuda_fail(nullptr, e, what);
    destroy_ctx(c);
    return r;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
  int prio_least = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&prio_least, &c->prio_high)) != cudaSuccess) return bail(e, "priority range");
  if ((e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, c->prio_high)) != cudaSuccess) return bail(e, "stream");
  for (cudaEvent_t *ev : {&c->ev_in, &c->ev_out, &c->ev_fork, &c->ev_join})
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "event");

  // geometry
  LbGeom &g = c->geo;
  g.nx = p.nx;
  g.ny = p.ny;
  g.nz = p.nz;
  g.ntx = L.ntx;
  g.V = (long long)p.nx * p.ny * p.nz;
  g.Vp = L.Vp;
  g.solid = (const uint32_t *)(c->ws + L.solid);
  g.tile_near = (const uint8_t *)(c->ws + L.tile);
  HostGeometry G;
  build_geometry(p, L.ntx, G);
  cudaStream_t s = c->user;
  if ((e = cudaMemcpyAsync(c->ws + L.solid, G.bits.data(), G.bits.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemcpyAsync(c->ws + L.tile, G.tile.data(), G.tile.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
  if ((e = cudaMemcpyAsync(c->ws + L.xslab, G.xslab.data(), G.xslab.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");

  c->phys.omega = (float)(1.0 / p.tau);
  c->phys.rho0 = (float)p.rho0;
  for (int a = 0; a < 3; ++a) c->phys.g[a] = (float)p.body_force[a];
  c->phys.forcing = p.forcing;

  // initial populations: (rho, u) staged in the second population buffer
  const float *drho = nullptr, *du = nullptr;
  std::vector<float> hfield;
  if (p.init_rho || p.init_u) {
    const size_t V = (size_t)g.V;
    hfield.assign(4 * V, 0.f);
    for (size_t k = 0; k < V; ++k) hfield[k] = p.init_rho ? (float)p.init_rho[k] : (float)p.rho0;
    for (size_t k = 0; k < 3 * V; ++k) hfield[V + k] = p.init_u ? (float)p.init_u[k] : 0.f;
    if ((e = cudaMemcpyAsync(c->pop[1], hfield.data(), hfield.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    drho = (const float *)c->pop[1];
    du = (const float *)c->pop[1] + V;
    if (!p.init_rho) drho = nullptr;
    if (!p.init_u) du = nullptr;
  }
  if ((e = launch_init_populations(p.storage, g, (float)p.rho0, drho, du, (float)p.init_tg_amp,
                                   c->pop[0], s)) != cudaSuccess)
    return bail(e, "init kernel");
  // the second buffer must hold zeros at solid nodes too: copy the first
  if ((e = cudaMemcpyAsync(c->pop[1], c->pop[0], (size_t)19 * L.Vp * store_bytes(p.storage), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return bail(e, "copy");

  // beads, in a local frame at the integer origin floor(r_0)
  DevStatus st{};
  st.t_transloc = -1;
  if ((e = cudaMemcpyAsync(c->status, &st, sizeof(st), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
  ChainArgs &a = c->chain;
  a.geo = g;
  a.xslab = (const uint8_t *)(c->ws + L.xslab);
  a.has_wall = p.wall_x >= 0;
  a.wall_x = p.wall_x;
  a.wall_t = p.wall_thickness;
  a.pore_d = p.wall_x >= 0 ? p.pore_d : 0;
  int y0 = 0, z0 = 0;
  if (p.wall_x >= 0) pore_origin(p, y0, z0);
  a.pore_y0 = y0;
  a.pore_z0 = z0;
  a.rho0 = (float)p.rho0;
  for (int k = 0; k < 3; ++k) a.g[k] = (float)p.body_force[k];
  a.forcing = p.forcing;
  a.coupling = p.coupling;
  a.N = p.n_beads;
  a.M = p.md_substeps;
  a.has_bonds = c->has_bonds;
  a.shake_maxit = p.shake_max_iter;
  a.dt = (float)(1.0 / std::max(p.md_substeps, 1));
  a.mass = (float)p.bead_mass;
  a.gamma = (float)p.gamma;
  a.kT = (float)p.kT;
  a.sigma = (float)p.lj_sigma;
  a.eps = (float)p.lj_eps;
  a.kappa = (float)p.kappa_phi;
  a.fdrive = (float)p.f_drive;
  a.shake_tol = (float)p.shake_tol;
  a.seed = p.seed;
  a.pos = (float4 *)(c->ws + L.pos);
  a.pos_lo = (float4 *)(c->ws + L.pos_lo);
  a.vel = (float4 *)(c->ws + L.vel);
  a.ui = (float4 *)(c->ws + L.ui);
  a.J = (float4 *)(c->ws + L.J);
  a.sp_node = (int *)(c->ws + L.sp_node);
  a.sp_w = (float *)(c->ws + L.sp_w);
  a.b0 = (const double *)(c->ws + L.b0);
  a.nl_cnt = (int *)(c->ws + L.nl_cnt);
  a.wl_cnt = (int *)(c->ws + L.wl_cnt);
  a.nl_list = (short *)(c->ws + L.nl_list);
  a.wl_list = (float4 *)(c->ws + L.wl_list);
  a.nl_ref = (float4 *)(c->ws + L.nl_ref);
  a.lam = (float *)(c->ws + L.lam);
  a.status = c->status;
  const int N = p.n_beads;
  // host staging kept alive until the stream synchronisation below
  std::vector<float4> hp(std::max(N, 1)), hl(std::max(N, 1)), hv(std::max(N, 1)),
      hz(std::max(N, 1), make_float4(0, 0, 0, 0));
  std::vector<double> hb(std::max(N - 1, 1), 0.0);
  if (N > 0) {
    a.ox = (int)std::floor(p.init_pos[0]);
    a.oy = (int)std::floor(p.init_pos[1]);
    a.oz = (int)std::floor(p.init_pos[2]);
    for (int i = 0; i < N; ++i) {
      // local coordinate split into a float hi part and the float remainder
      const double lx = p.init_pos[3 * i] - a.ox, ly = p.init_pos[3 * i + 1] - a.oy,
                   lz = p.init_pos[3 * i + 2] - a.oz;
      hp[i] = make_float4((float)lx, (float)ly, (float)lz, 0.f);
      hl[i] = make_float4((float)(lx - (double)hp[i].x), (float)(ly - (double)hp[i].y),
                          (float)(lz - (double)hp[i].z), 0.f);
      hv[i] = p.init_vel ? make_float4((float)p.init_vel[3 * i], (float)p.init_vel[3 * i + 1],
                                       (float)p.init_vel[3 * i + 2], 0.f)
                         : make_float4(0, 0, 0, 0);
    }
    for (int k = 0; k + 1 < N; ++k)
      hb[k] = p.n_constraints > 0 ? p.bond_len[k] : p.bond_length;
    if ((e = cudaMemcpyAsync(a.pos, hp.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemcpyAsync(a.pos_lo, hl.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemcpyAsync(a.vel, hv.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemcpyAsync(a.ui, hz.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemcpyAsync(a.J, hz.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemcpyAsync(c->ws + L.b0, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = cudaMemsetAsync(a.sp_node, 0xff, 8 * (size_t)N * sizeof(int), s)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(a.nl_cnt, 0, (size_t)N * sizeof(int), s)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(a.wl_cnt, 0, (size_t)N * sizeof(int), s)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(a.lam, 0, (size_t)N * sizeof(float), s)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemcpyAsync(a.nl_ref, hp.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s)) != cudaSuccess) return bail(e, "upload");
    if ((e = md_prepare(N)) != cudaSuccess) return bail(e, "md attributes");
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "create sync");
  *out = c;
  return LBMD_OK;
}

int lbmd_step(lbmd_ctx *c, int64_t n_steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_steps < 0) return fail(LBMD_EINVAL, "n_steps < 0");
  if (n_steps == 0) return LBMD_OK;
  CK(c, cudaEventRecord(c->ev_in, c->user));
  CK(c, cudaStreamWaitEvent(c->own, c->ev_in, 0));
  if (c->timing) {
    for (int64_t k = 0; k < n_steps; ++k) {
      CK(c, enqueue_step(c, c->cur));
      c->cur ^= 1;
    }
  } else {
    int64_t left = n_steps;
    for (int gi = 2; gi >= 0; --gi) {
      const int len = kGraphSteps[gi];
      while (left >= len) {
        if (!c->graph[c->cur][gi]) CK(c, capture(c, c->cur, len, &c->graph[c->cur][gi]));
        CK(c, cudaGraphLaunch(c->graph[c->cur][gi], c->own));
        if (len & 1) c->cur ^= 1;
        left -= len;
      }
    }
  }
  CK(c, cudaEventRecord(c->ev_out, c->own));
  CK(c, cudaStreamWaitEvent(c->user, c->ev_out, 0));
  return LBMD_OK;
}

int lbmd_read_fields(lbmd_ctx *c, float *rho, float *u, int dst_is_device) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!rho && !u) return LBMD_OK;
  const LbGeom &g = c->geo;
  const void *src = c->pop[c->cur];
  if (dst_is_device) {
    CK(c, launch_read_moments(c->p.storage, g, c->phys, src, 0, g.nz, rho, u, g.V, c->user));
    return LBMD_OK;
  }
  const long long plane = (long long)g.nx * g.ny;
  const long long nzc_max = std::max(1LL, c->L.chunk_cells / plane);
  float *srho = c->stage, *su = c->stage + nzc_max * plane;
  for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
    const long long nzc = std::min(nzc_max, (long long)g.nz - z0);
    const long long cells = nzc * plane;
    CK(c, launch_read_moments(c->p.storage, g, c->phys, src, z0, nzc, rho ? srho : nullptr,
                              u ? su : nullptr, cells, c->user));
    if (rho)
      CK(c, cudaMemcpyAsync(rho + z0 * plane, srho, cells * 4, cudaMemcpyDeviceToHost, c->user));
    if (u)
      for (int a = 0; a < 3; ++a)
        CK(c, cudaMemcpyAsync(u + a * g.V + z0 * plane, su + a * cells, cells * 4,
                              cudaMemcpyDeviceToHost, c->user));
  }
  CK(c, cudaStreamSynchronize(c->user));
  return LBMD_OK;
}

int lbmd_read_populations(lbmd_ctx *c, float *f, int dst_is_device) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!f) return fail(LBMD_EINVAL, "f is NULL");
  const LbGeom &g = c->geo;
  const void *src = c->pop[c->cur];
  if (dst_is_device) {
    CK(c, launch_read_pulled(c->p.storage, g, (float)c->p.rho0, src, 0, g.nz, f, g.V, c->user));
    return LBMD_OK;
  }
  const long long plane = (long long)g.nx * g.ny;
  const long long nzc_max = std::max(1LL, c->L.chunk_cells / plane);
  for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
    const long long nzc = std::min(nzc_max, (long long)g.nz - z0);
    const long long cells = nzc * plane;
    CK(c, launch_read_pulled(c->p.storage, g, (float)c->p.rho0, src, z0, nzc, c->stage, cells, c->user));
    for (int q = 0; q < 19; ++q)
      CK(c, cudaMemcpyAsync(f + q * g.V + z0 * plane, c->stage + q * cells, cells * 4,
                            cudaMemcpyDeviceToHost, c->user));
  }
  CK(c, cudaStreamSynchronize(c->user));
  return LBMD_OK;
}

static int read_bead_pair(lbmd_ctx *c, double *x, double *y, int dst_is_device, bool aux) {
  int rc = check_ctx(c);
  if (rc) return rc;
  const int N = c->N;
  if (N == 0 || (!x && !y)) return LBMD_OK;
  const ChainArgs &a = c->chain;
  double *dx = x, *dy = y;
  if (!dst_is_device) {
    dx = x ? (double *)c->stage : nullptr;
    dy = y ? (double *)c->stage + 3 * N : nullptr;
  }
  if (aux)
    CK(c, launch_read_bead_aux(a.ui, a.J, N, dx, dy, c->user));
  else
    CK(c, launch_read_beads(a.pos, a.pos_lo, a.vel, N, a.ox, a.oy, a.oz, dx, dy, c->user));
  if (!dst_is_device) {
    if (x) CK(c, cudaMemcpyAsync(x, dx, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->user));
    if (y) CK(c, cudaMemcpyAsync(y, dy, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->user));
    CK(c, cudaStreamSynchronize(c->user));
  }
  return LBMD_OK;
}

int lbmd_read_beads(lbmd_ctx *c, double *pos, double *vel, int dst_is_device) {
  return read_bead_pair(c, pos, vel, dst_is_device, false);
}

int lbmd_read_bead_aux(lbmd_ctx *c, double *u_i, double *impulse, int dst_is_device) {
  return read_bead_pair(c, u_i, impulse, dst_is_device, true);
}

int lbmd_status(lbmd_ctx *c, int64_t *step, int32_t *n_trans, int32_t *state, int64_t *t_transloc) {
  int rc = check_ctx(c);
  if (rc) return rc;
  DevStatus st;
  CK(c, cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->user));
  CK(c, cudaStreamSynchronize(c->user));
  if (step) *step = st.step;
  if (n_trans) *n_trans = st.n_trans;
  if (state) *state = st.state;
  if (t_transloc) *t_transloc = st.t_transloc;
  return LBMD_OK;
}

int lbmd_solver_stats(lbmd_ctx *c, int32_t *newton_iters_last_step, int32_t *failed_steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  DevStatus st;
  CK(c, cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->user));
  CK(c, cudaStreamSynchronize(c->user));
  if (newton_iters_last_step) *newton_iters_last_step = st.newton_iters;
  if (failed_steps) *failed_steps = st.shake_fail;
  return LBMD_OK;
}

int lbmd_set_kernel_timing(lbmd_ctx *c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(c, cudaStreamSynchronize(c->own));
  c->timing = enable ? 1 : 0;
  c->tev_used = 0;
  c->timed_ms[0] = c->timed_ms[1] = c->timed_ms[2] = 0;
  c->timed_count = 0;
  return LBMD_OK;
}

static int collect_times(lbmd_ctx *c) {
  CK(c, cudaStreamSynchronize(c->own));
  CK(c, cudaStreamSynchronize(c->side));
  for (size_t k = 0; k + 5 < c->tev_used; k += 6) {
    for (int q = 0; q < 3; ++q) {
      float ms = 0.f;
      CK(c, cudaEventElapsedTime(&ms, c->tev[k + 2 * q], c->tev[k + 2 * q + 1]));
      c->timed_ms[q] += ms;
    }
    c->timed_count += 1;
  }
  c->tev_used = 0;
  return LBMD_OK;
}

int lbmd_lb_kernel_time(lbmd_ctx *c, double *total_ms, int64_t *launches) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = collect_times(c))) return rc;
  if (total_ms) *total_ms = c->timed_ms[0];
  if (launches) *launches = c->timed_count;
  return LBMD_OK;
}

int lbmd_kernel_times(lbmd_ctx *c, double *lb_ms, double *md_ms, double *spread_ms,
                      int64_t *steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = collect_times(c))) return rc;
  if (lb_ms) *lb_ms = c->timed_ms[0];
  if (md_ms) *md_ms = c->timed_ms[1];
  if (spread_ms) *spread_ms = c->timed_ms[2];
  if (steps) *steps = c->timed_count;
  return LBMD_OK;
}

int lbmd_destroy(lbmd_ctx *c) {
  if (!c) return LBMD_OK;
  cudaStreamSynchronize(c->own);
  cudaStreamSynchronize(c->side);
  destroy_ctx(c);
  return LBMD_OK;
}

}  // extern "C"

