// lbmd_host.cu -- host-side setup of one box (parameter checks, workspace
// layout, the Sec. III geometry, the initial state), shared by the
// single-box context and the ensemble.  No device memory is allocated here.
#include "lbmd_host.h"

#include "lbmd_common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace lbmd {

namespace {
thread_local char g_msg[512] = "";
}  // namespace

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

const char *last_message() { return g_msg; }

bool params_have_bonds(const lbmd_params &p) {
  return p.n_constraints == -1 ? p.n_beads > 1 : p.n_constraints > 0;
}

long long chunk_cells_for(const lbmd_params &p) {
  const long long V = (long long)p.nx * p.ny * p.nz;
  const long long plane = (long long)p.nx * p.ny;
  long long c = std::min(V, std::max(plane, (long long)(1 << 20)));
  c = (c / plane) * plane;  // whole z-planes
  return c < plane ? plane : c;
}

size_t stage_floats_for(const lbmd_params &p) {
  const size_t Np = (size_t)std::max(p.n_beads, 1);
  // 19 populations of a chunk, or 6 N doubles of bead read-out plus a status word
  return std::max((size_t)19 * (size_t)chunk_cells_for(p), (size_t)6 * Np * 2 + 8);
}

Layout make_layout(const lbmd_params &p, bool single_box) {
  Layout L{};
  const long long V = (long long)p.nx * p.ny * p.nz;
  L.Vp = (V + 63) / 64 * 64;
  L.ntx = (p.nx + 31) / 32;
  const size_t rows = (size_t)p.ny * p.nz;
  const size_t Np = (size_t)std::max(p.n_beads, 1);
  L.chunk_cells = chunk_cells_for(p);
  L.stage_floats = single_box ? stage_floats_for(p) : 0;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.popA = take((size_t)19 * L.Vp * store_bytes(p.storage));
  // in-place streaming keeps a single population buffer
  L.popB = p.streaming == LBMD_STREAM_AA ? L.popA : take((size_t)19 * L.Vp * store_bytes(p.storage));
  L.solid = take(rows * L.ntx * sizeof(uint32_t));
  L.tile = take(rows * L.ntx);
  L.lmask = take((size_t)V * sizeof(uint32_t));
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
  L.diag = take((size_t)std::max(p.diag_capacity, 0) * sizeof(DevDiag));
  // a chain coupled to the solvent: the spread owner of every node (4 bytes
  // per node) and the fixed-point sums of the 8 N transfer entries; a single
  // box also keeps the apply records of the entries
  const bool coupled = p.n_beads > 0 && !p.solvent_free;
  L.owner = coupled ? take((size_t)V * sizeof(int)) : 0;
  L.acc = coupled ? take(8 * Np * sizeof(SpreadAcc)) : 0;
  L.sp_src = coupled && single_box ? take(8 * Np * sizeof(float4)) : 0;
  L.stage = single_box ? take(L.stage_floats * sizeof(float)) : 0;
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
  if (p->solvent_free != 0 && p->solvent_free != 1)
    return fail(LBMD_EINVAL, "solvent_free must be 0 or 1");
  if (p->solvent_free && p->n_beads < 1) return fail(LBMD_EINVAL, "solvent_free needs n_beads >= 1");
  if (p->streaming != LBMD_STREAM_PULL && p->streaming != LBMD_STREAM_AA)
    return fail(LBMD_EINVAL, "unknown streaming %d", p->streaming);
  if (!(p->kT_fluid >= 0) || !std::isfinite(p->kT_fluid))
    return fail(LBMD_EINVAL, "kT_fluid must be >= 0");
  if (p->diag_every < 0 || p->diag_capacity < 0)
    return fail(LBMD_EINVAL, "diag_every and diag_capacity must be >= 0");
  if (p->diag_every > 0 && (p->n_beads < 1 || p->diag_capacity < 1))
    return fail(LBMD_EINVAL, "diag_every > 0 needs n_beads >= 1 and diag_capacity >= 1");
  if (p->y_walls && p->ny < 3) return fail(LBMD_EINVAL, "y_walls needs ny >= 3");
  if (p->n_beads < 0 || p->n_beads > LBMD_MAX_BEADS)
    return fail(LBMD_EINVAL, "n_beads must be in [0, %d]", LBMD_MAX_BEADS);
  if (p->n_beads > 0) {
    if (p->md_substeps < 1 || p->md_substeps > 255)
      return fail(LBMD_EINVAL, "md_substeps must be in [1, 255]");
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
    if (params_have_bonds(*p) && (p->shake_max_iter < 1 || !(p->shake_tol > 0)))
      return fail(LBMD_EINVAL, "shake_max_iter >= 1 and shake_tol > 0 required");
    if (p->init_pos)
      for (int i = 0; i < 3 * p->n_beads; ++i)
        if (!std::isfinite(p->init_pos[i])) return fail(LBMD_EINVAL, "init_pos not finite");
  }
  return LBMD_OK;
}

static void pore_origin(const lbmd_params &p, int &y0, int &z0) {
  y0 = p.pore_y0 >= 0 ? p.pore_y0 : (p.ny - p.pore_d) / 2;
  z0 = p.pore_z0 >= 0 ? p.pore_z0 : (p.nz - p.pore_d) / 2;
}

// Solid nodes of Sec. III: the wall layers minus the centred pore, plus the
// optional rows y = 0 and y = ny - 1.
static bool is_solid(const lbmd_params &p, int x, int y, int z) {
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

// Seeded start (Sec. III; reading of the walk: bead 0 at the pore mouth,
// x_w + t at the pore centre, bead 1 one bond further along +x, every later
// bead one bond in a uniformly random direction from the previous one,
// rejected if it comes within 2^(1/6) sigma of a bead two or more places
// away along the chain (minimum image), of a solid node, or of the wall plane
// (x < x_w + t - 1 + 2^(1/6) sigma), or beyond x_w + n_x - 2^(1/6) sigma;
// after 1000 rejections of one bead the walk restarts).  Random numbers:
// Philox4x32-10 keyed by the seed, counter (bead, attempt, restart, 1 << 8)
// -- stream 1, beside the bead noise (stream 0) and the fluid noise
// (stream 2); direction from two uniforms: cos(theta) = 2 u1 - 1,
// phi = 2 pi u2.
int seeded_start(const lbmd_params &p, std::vector<double> &pos) {
  const int N = p.n_beads;
  pos.assign(3 * (size_t)std::max(N, 0), 0.0);
  if (N <= 0) return LBMD_OK;
  const double rc = 1.122462048309373 * p.lj_sigma, rc2 = rc * rc;
  const double L[3] = {(double)p.nx, (double)p.ny, (double)p.nz};
  auto bond = [&](int k) {  // length of the bond (k, k + 1)
    if (p.n_constraints > 0) return p.bond_len[k];
    return p.bond_length > 0 ? p.bond_length : rc;
  };
  double start[3], x_lo = -INFINITY, x_hi = INFINITY;
  const int t = p.wall_thickness;
  if (p.wall_x >= 0) {
    int y0, z0;
    pore_origin(p, y0, z0);
    start[0] = p.wall_x + t;
    start[1] = y0 + 0.5 * (p.pore_d - 1);
    start[2] = z0 + 0.5 * (p.pore_d - 1);
    x_lo = p.wall_x + t - 1 + rc;
    x_hi = p.wall_x + L[0] - rc;
  } else {
    for (int a = 0; a < 3; ++a) start[a] = 0.5 * L[a];
  }
  auto min_image = [&](double d, int a) { return d - L[a] * std::floor(d / L[a] + 0.5); };
  auto near_solid = [&](const double *r) {
    if (p.wall_x < 0 && !p.y_walls) return false;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = (int)std::ceil(r[a] - rc);
      hi[a] = (int)std::floor(r[a] + rc);
    }
    for (int x = lo[0]; x <= hi[0]; ++x)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int z = lo[2]; z <= hi[2]; ++z) {
          const double dx = x - r[0], dy = y - r[1], dz = z - r[2];
          if (dx * dx + dy * dy + dz * dz >= rc2) continue;
          const int wx = ((x % p.nx) + p.nx) % p.nx, wy = ((y % p.ny) + p.ny) % p.ny,
                    wz = ((z % p.nz) + p.nz) % p.nz;
          if (is_solid(p, wx, wy, wz)) return true;
        }
    return false;
  };
  const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
  for (uint32_t restart = 0; restart < 1000; ++restart) {
    for (int a = 0; a < 3; ++a) pos[a] = start[a];
    if (N > 1) {
      pos[3] = start[0] + bond(0);
      pos[4] = start[1];
      pos[5] = start[2];
    }
    bool ok = true;
    for (int i = 2; i < N && ok; ++i) {
      const double b = bond(i - 1);
      bool placed = false;
      for (uint32_t attempt = 0; attempt < 1000 && !placed; ++attempt) {
        const U4 r = philox4x32_10(U4{(uint32_t)i, attempt, restart, 1u << 8}, k0, k1);
        const double u1 = ((r.x >> 9) + 0.5) * 0x1p-23, u2 = ((r.y >> 9) + 0.5) * 0x1p-23;
        const double ct = 2.0 * u1 - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
        const double ph = 2.0 * M_PI * u2;
        double c[3] = {pos[3 * (i - 1)] + b * st * std::cos(ph), pos[3 * (i - 1) + 1] + b * st * std::sin(ph),
                       pos[3 * (i - 1) + 2] + b * ct};
        if (!(c[0] >= x_lo && c[0] <= x_hi)) continue;
        bool clash = false;
        for (int j = 0; j + 1 < i && !clash; ++j) {
          const double dx = min_image(c[0] - pos[3 * j], 0), dy = min_image(c[1] - pos[3 * j + 1], 1),
                       dz = min_image(c[2] - pos[3 * j + 2], 2);
          clash = dx * dx + dy * dy + dz * dz < rc2;
        }
        if (clash || near_solid(c)) continue;
        for (int a = 0; a < 3; ++a) pos[3 * i + a] = c[a];
        placed = true;
      }
      ok = placed;
    }
    if (ok) return LBMD_OK;
  }
  return fail(LBMD_EINVAL, "no self-avoiding chain start of %d beads fits the box", N);
}

namespace {
struct HostGeometry {
  std::vector<uint32_t> bits;   // [nz][ny][ntx]
  std::vector<uint8_t> tile;    // [nz][ny][ntx]
};

}  // namespace

static void build_geometry(const lbmd_params &p, int ntx, HostGeometry &G) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  G.bits.assign((size_t)nz * ny * ntx, 0u);
  G.tile.assign((size_t)nz * ny * ntx, 0u);
  const bool any_solid = p.y_walls || p.wall_x >= 0;
  if (!any_solid) return;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        if (is_solid(p, x, y, z)) {
          G.bits[((size_t)z * ny + y) * ntx + (x >> 5)] |= 1u << (x & 31);
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


int copy_diagnostics(const DevStatus *status, const DevDiag *diag, int cap, lbmd_diag *records,
                     int32_t max_records, int32_t *n_records, cudaStream_t s) {
  if (max_records < 0 || (max_records > 0 && !records))
    return fail(LBMD_EINVAL, "records is NULL or max_records < 0");
  DevStatus st;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(LBMD_ECUDA, "diagnostics: %s", cudaGetErrorString(e));
  const int n = std::min(std::min(st.diag_count, cap), max_records);
  std::vector<DevDiag> h((size_t)std::max(n, 1));
  if (n > 0 && ((e = cudaMemcpyAsync(h.data(), diag, n * sizeof(DevDiag), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess))
    return fail(LBMD_ECUDA, "diagnostics: %s", cudaGetErrorString(e));
  for (int k = 0; k < n; ++k) {
    lbmd_diag &r = records[k];
    r.step = h[k].step;
    r.n_trans = h[k].n_trans;
    r.reserved = 0;
    r.r_u = h[k].r_u;
    r.r_t = h[k].r_t;
    r.r_e = h[k].r_e;
    r.s_h = h[k].s_h;
    r.s_e = h[k].s_e;
    r.kinetic = h[k].kinetic;
  }
  if (n_records) *n_records = std::min(st.diag_count, cap);
  return LBMD_OK;
}

cudaError_t init_instance(const lbmd_params &p, const Layout &L, char *ws, cudaStream_t s,
                          Instance &out, const char **what) {
  cudaError_t e;
#define UP(call, msg)                   \
  do {                                  \
    if ((e = (call)) != cudaSuccess) {  \
      *what = msg;                      \
      return e;                         \
    }                                   \
  } while (0)
  out = Instance{};
  out.pop[0] = ws + L.popA;
  out.pop[1] = ws + L.popB;
  out.status = (DevStatus *)(ws + L.status);
  out.has_bonds = params_have_bonds(p) ? 1 : 0;

  // geometry
  LbGeom &g = out.geo;
  g.nx = p.nx;
  g.ny = p.ny;
  g.nz = p.nz;
  g.ntx = L.ntx;
  g.V = (long long)p.nx * p.ny * p.nz;
  g.Vp = L.Vp;
  g.solid = (const uint32_t *)(ws + L.solid);
  g.tile_near = (const uint8_t *)(ws + L.tile);
  g.lmask = (const uint32_t *)(ws + L.lmask);
  HostGeometry G;
  build_geometry(p, L.ntx, G);
  UP(cudaMemcpyAsync(ws + L.solid, G.bits.data(), G.bits.size() * 4, cudaMemcpyHostToDevice, s), "upload");
  UP(cudaMemcpyAsync(ws + L.tile, G.tile.data(), G.tile.size(), cudaMemcpyHostToDevice, s), "upload");
  UP(launch_link_mask(g, (uint32_t *)(ws + L.lmask), s), "link mask");

  out.phys.omega = (float)(1.0 / p.tau);
  out.phys.rho0 = (float)p.rho0;
  for (int a = 0; a < 3; ++a) out.phys.g[a] = (float)p.body_force[a];
  out.phys.forcing = p.forcing;
  out.phys.seed = p.seed;
  out.phys.step = nullptr;
  out.phys.nonfinite = &out.status->pop_bad;
  for (int k = 0; k < 15; ++k) out.phys.fl_amp[k] = 0.f;
  if (p.kT_fluid > 0) {
    fluct_amplitudes(p.kT_fluid, p.tau, out.phys.fl_amp);
    out.phys.step = &out.status->step;
  }

  // initial populations
  std::vector<float> hfield;
  if (p.init_rho || p.init_u) {
    const size_t V = (size_t)g.V;
    hfield.assign(4 * V, 0.f);
    for (size_t k = 0; k < V; ++k) hfield[k] = p.init_rho ? (float)p.init_rho[k] : (float)p.rho0;
    for (size_t k = 0; k < 3 * V; ++k) hfield[V + k] = p.init_u ? (float)p.init_u[k] : 0.f;
  }
  if (p.streaming == LBMD_STREAM_AA) {
    // one buffer, f_eq stored locally; given fields go through the staging
    // buffer (19 floats per cell of a chunk) one z-slab at a time
    if (hfield.empty()) {
      UP(launch_init_local(p.storage, g, (float)p.rho0, nullptr, nullptr, 0, (float)p.init_tg_amp, 0,
                           g.nz, out.pop[0], s),
         "init kernel");
    } else {
      if (L.stage_floats == 0) {
        *what = "in-place streaming with initial fields needs the staging buffer";
        return cudaErrorInvalidValue;
      }
      const long long plane = (long long)g.nx * g.ny;
      const long long nzc_max = std::max(1LL, L.chunk_cells / plane);
      float *st = (float *)(ws + L.stage);
      for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
        const long long nzc = std::min(nzc_max, (long long)g.nz - z0), cells = nzc * plane;
        for (int a = 0; a < 4; ++a)
          UP(cudaMemcpyAsync(st + a * cells, hfield.data() + a * (size_t)g.V + z0 * plane, cells * 4,
                             cudaMemcpyHostToDevice, s),
             "upload");
        UP(launch_init_local(p.storage, g, (float)p.rho0, p.init_rho ? st : nullptr,
                             p.init_u ? st + cells : nullptr, cells, (float)p.init_tg_amp, z0, nzc,
                             out.pop[0], s),
           "init kernel");
      }
    }
  } else {
    // (rho, u) staged in the second population buffer
    const float *drho = nullptr, *du = nullptr;
    if (!hfield.empty()) {
      UP(cudaMemcpyAsync(out.pop[1], hfield.data(), hfield.size() * 4, cudaMemcpyHostToDevice, s), "upload");
      drho = p.init_rho ? (const float *)out.pop[1] : nullptr;
      du = p.init_u ? (const float *)out.pop[1] + g.V : nullptr;
    }
    UP(launch_init_populations(p.storage, g, (float)p.rho0, drho, du, (float)p.init_tg_amp, out.pop[0], s),
       "init kernel");
    // the second buffer must hold zeros at solid nodes too: copy the first
    UP(cudaMemcpyAsync(out.pop[1], out.pop[0], (size_t)19 * L.Vp * store_bytes(p.storage),
                       cudaMemcpyDeviceToDevice, s),
       "copy");
  }

  // beads, in a local frame at the integer origin floor(r_0)
  DevStatus st{};
  st.t_transloc = -1;
  UP(cudaMemcpyAsync(out.status, &st, sizeof(st), cudaMemcpyHostToDevice, s), "upload");
  ChainArgs &a = out.chain;
  a = ChainArgs{};
  const size_t ne = 8 * (size_t)std::max(p.n_beads, 1);
  if (L.sp_src) {
    // apply records without a node (-1)
    a.sp_src = (float4 *)(ws + L.sp_src);
    UP(cudaMemsetAsync(a.sp_src, 0xff, ne * sizeof(float4), s), "memset");
  }
  if (L.owner) {
    // spread owners at rest (every byte 0x7f = kOwnerFree), impulse sums zero
    a.owner = (int *)(ws + L.owner);
    a.acc = (SpreadAcc *)(ws + L.acc);
    UP(cudaMemsetAsync(a.owner, 0x7f, (size_t)g.V * sizeof(int), s), "memset");
    UP(cudaMemsetAsync(a.acc, 0, ne * sizeof(SpreadAcc), s), "memset");
  }
  a.geo = g;
  a.has_wall = p.wall_x >= 0;
  a.wall_x = p.wall_x;
  a.wall_t = p.wall_thickness;
  a.pore_d = p.wall_x >= 0 ? p.pore_d : 0;
  int y0 = 0, z0 = 0;
  if (p.wall_x >= 0) pore_origin(p, y0, z0);
  a.pore_y0 = y0;
  a.pore_z0 = z0;
  a.y_walls = p.y_walls;
  a.rho0 = (float)p.rho0;
  for (int k = 0; k < 3; ++k) a.g[k] = (float)p.body_force[k];
  a.forcing = p.forcing;
  a.coupling = p.coupling;
  a.N = p.n_beads;
  a.M = p.md_substeps;
  a.has_bonds = out.has_bonds;
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
  a.pos = (float4 *)(ws + L.pos);
  a.pos_lo = (float4 *)(ws + L.pos_lo);
  a.vel = (float4 *)(ws + L.vel);
  a.ui = (float4 *)(ws + L.ui);
  a.J = (float4 *)(ws + L.J);
  a.sp_node = (int *)(ws + L.sp_node);
  a.sp_w = (float *)(ws + L.sp_w);
  a.b0 = (const double *)(ws + L.b0);
  a.nl_cnt = (int *)(ws + L.nl_cnt);
  a.wl_cnt = (int *)(ws + L.wl_cnt);
  a.nl_list = (short *)(ws + L.nl_list);
  a.wl_list = (float4 *)(ws + L.wl_list);
  a.nl_ref = (float4 *)(ws + L.nl_ref);
  a.lam = (float *)(ws + L.lam);
  a.status = out.status;
  a.diag = (DevDiag *)(ws + L.diag);
  a.diag_every = p.diag_every;
  a.diag_cap = p.diag_capacity;
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
    for (int k = 0; k + 1 < N; ++k) hb[k] = p.n_constraints > 0 ? p.bond_len[k] : p.bond_length;
    UP(cudaMemcpyAsync(a.pos, hp.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemcpyAsync(a.pos_lo, hl.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemcpyAsync(a.vel, hv.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemcpyAsync(a.ui, hz.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemcpyAsync(a.J, hz.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemcpyAsync(ws + L.b0, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, s), "upload");
    UP(cudaMemsetAsync(a.sp_node, 0xff, 8 * (size_t)N * sizeof(int), s), "memset");
    UP(cudaMemsetAsync(a.nl_cnt, 0, (size_t)N * sizeof(int), s), "memset");
    UP(cudaMemsetAsync(a.wl_cnt, 0, (size_t)N * sizeof(int), s), "memset");
    UP(cudaMemsetAsync(a.lam, 0, (size_t)N * sizeof(float), s), "memset");
    UP(cudaMemcpyAsync(a.nl_ref, hp.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s), "upload");
    UP(md_prepare(), "md attributes");
  }
  UP(cudaStreamSynchronize(s), "create sync");
#undef UP
  return cudaSuccess;
}

}  // namespace lbmd
