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

#include "lbmd_host.h"

using namespace lbmd;

// ---------------------------------------------------------------------------
struct lbmd_ctx {
  lbmd_params p;  // host pointers cleared after create
  Layout L;
  LbGeom geo;
  LbPhys phys;
  ChainArgs chain;
  char *ws;
  char *pop[2];  // equal with in-place streaming
  int cur;  // pull: pop[cur] holds the post-collision populations of the last
            // step; in place: 0 = kPopAALocal, 1 = kPopAASwap
  int aa;   // in-place (AA-pattern) streaming
  int N, has_bonds;
  cudaStream_t user;        // caller's stream
  cudaStream_t own, side;   // private streams: steps run on own, MD on side
  int prio_high;            // greatest stream priority of the device
  cudaEvent_t ev_in, ev_out, ev_fork, ev_join;
  cudaGraphExec_t graph[2][3];  // [starting buffer][1, 2, kBlockSteps steps]
  // one step followed by the bead-block read-out, per starting buffer
  // (lbmd_step_read_async); the read-out node's destination is set per launch
  cudaGraph_t rtmpl[2];
  cudaGraphExec_t rgraph[2];
  cudaGraphNode_t rnode[2];
  cudaKernelNodeParams rparams[2];
  int sticky;
  int timing;
  std::vector<cudaEvent_t> tev;  // per timed step: lb, md, spread start/stop pairs
  size_t tev_used;
  std::vector<cudaGraphExec_t> tgraphs;  // graphs of timed steps, destroyed once collected
  double timed_ms[3];            // summed durations of stream-collide, MD, spread
  long long timed_count;
  DevStatus *status;
  float *stage;
  // pinned host staging of the host bead read-outs (with the status word,
  // so that lbmd_status right after needs no second synchronisation)
  char *pinned;
  DevStatus status_cache;
  int status_fresh;  // status_cache is current: no step enqueued since
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

// Layout (kPop*) of the populations when the context's `cur` is `src`.
int pop_mode(const lbmd_ctx *c, int src) {
  return c->aa ? (src ? kPopAASwap : kPopAALocal) : kPopPull;
}

// A timing event: captured into a step graph as an event-record node, so that
// the recorded times are those of the graph's execution.
cudaError_t record_timing(cudaEvent_t ev, cudaStream_t s) {
  return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
}

// Enqueue one coupled LB step reading pop[src] and writing pop[1 - src] (with
// in-place streaming: the one buffer, even step if src = 0, odd if 1) on the
// private stream `own`: the MD cycle (gather + M substeps) on the side stream
// concurrently with the stream-collide, then the spread of the bead impulses
// into the new post-collision populations.  With paper forcing the bead source
// does not depend on f, so adding it after the collision is exact.
cudaError_t enqueue_step(lbmd_ctx *c, int src) {
  const void *A = c->pop[src];
  void *B = c->pop[1 - src];
  const int mode_out = pop_mode(c, 1 - src);
  cudaError_t e;
  cudaEvent_t t[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (c->timing) {
    // events reserved by lbmd_step before the capture
    if (c->tev_used + 6 > c->tev.size()) return cudaErrorInvalidValue;
    for (int k = 0; k < 6; ++k) t[k] = c->tev[c->tev_used + k];
    c->tev_used += 6;
  }
  if (c->p.solvent_free) {
    // no solvent (u_i stays 0): the M MD substeps, then the spread, which
    // finds no transfer node and only advances the step counter
    if (t[2] && (e = record_timing(t[2], c->own)) != cudaSuccess) return e;
    if ((e = launch_md_cycle(c->chain, c->prio_high, c->own)) != cudaSuccess) return e;
    if (t[3] && (e = record_timing(t[3], c->own)) != cudaSuccess) return e;
    for (int k : {0, 1, 4})
      if (t[k] && (e = record_timing(t[k], c->own)) != cudaSuccess) return e;
    if ((e = launch_spread_apply(c->p.storage, c->geo, c->chain, B, mode_out, false, c->status,
                                 c->own)) != cudaSuccess)
      return e;
    if (t[5] && (e = record_timing(t[5], c->own)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  // Where the owners' sums are converted: when the MD branch sets the step,
  // in the apply (one launch fewer on that branch); when the stream-collide
  // sets it, beside it in k_spread_finalize, keeping the apply after it short.
  const bool take = spread_take_in_apply(c->p.storage, c->geo.V);
  if (c->N > 0) {
    // (1) gather from the pre-step populations, and the MD cycle on the
    // high-priority side stream while the stream-collide runs on the main
    // one.  Where the stream-collide sets the step, the gather runs on the
    // side stream too, so the stream-collide starts at once (FP32 benchmark
    // box: 113.5 -> 111.5 us); where the MD branch sets it, the gather runs
    // first, before the stream-collide takes the SMs (FP16: 83.7 against
    // 85.6 us the other way).
    ChainArgs a = c->chain;
    a.f = A;
    a.f_mode = pop_mode(c, src);
    const bool gather_beside = !take;
    cudaStream_t gs = gather_beside ? c->side : c->own;
    if (gather_beside) {
      if ((e = cudaEventRecord(c->ev_fork, c->own)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c->side, c->ev_fork, 0)) != cudaSuccess) return e;
    }
    if (t[2] && (e = record_timing(t[2], gs)) != cudaSuccess) return e;
    if ((e = launch_gather(c->p.storage, a, gs)) != cudaSuccess) return e;
    if (!gather_beside) {
      if ((e = cudaEventRecord(c->ev_fork, c->own)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c->side, c->ev_fork, 0)) != cudaSuccess) return e;
    }
    if ((e = launch_md_cycle(a, c->prio_high, c->side)) != cudaSuccess) return e;
    if (t[3] && (e = record_timing(t[3], c->side)) != cudaSuccess) return e;
    // sum part of the spread, beside the stream-collide
    if ((e = launch_spread_sum(c->chain, !take, c->side)) != cudaSuccess) return e;
  } else if (t[2]) {
    if ((e = record_timing(t[2], c->own)) != cudaSuccess) return e;
    if ((e = record_timing(t[3], c->own)) != cudaSuccess) return e;
  }
  if (t[0] && (e = record_timing(t[0], c->own)) != cudaSuccess) return e;
  DevStatus *bump = c->N > 0 ? nullptr : c->status;
  if (c->phys.step) {
    // thermal source: the kernel reads the step count, so a box without
    // beads advances it in a separate launch afterwards
    e = c->aa ? launch_lb_aa_fluct(c->p.storage, c->geo, c->phys, B, src, c->own)
              : launch_lb_stream_collide_fluct(c->p.storage, c->geo, c->phys, A, B, c->own);
    if (e != cudaSuccess) return e;
    if (c->N == 0 && (e = launch_bump_step(c->status, c->own)) != cudaSuccess) return e;
  } else {
    e = c->aa ? launch_lb_aa(c->p.storage, c->geo, c->phys, B, src, bump, c->own)
              : launch_lb_stream_collide(c->p.storage, c->geo, c->phys, A, B, bump, c->own);
    if (e != cudaSuccess) return e;
  }
  if (t[1] && (e = record_timing(t[1], c->own)) != cudaSuccess) return e;
  if (c->N > 0) {
    if ((e = cudaEventRecord(c->ev_join, c->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->own, c->ev_join, 0)) != cudaSuccess) return e;
    if (t[4] && (e = record_timing(t[4], c->own)) != cudaSuccess) return e;
    if ((e = launch_spread_apply(c->p.storage, c->geo, c->chain, B, mode_out, take, c->status,
                                 c->own)) != cudaSuccess)
      return e;
    if (t[5] && (e = record_timing(t[5], c->own)) != cudaSuccess) return e;
  } else if (t[4]) {
    if ((e = record_timing(t[4], c->own)) != cudaSuccess) return e;
    if ((e = record_timing(t[5], c->own)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Bytes from the start of the bead positions to the end of the velocities.
size_t bead_span(const lbmd_ctx *c) {
  return c->L.vel - c->L.pos + (size_t)std::max(c->N, 1) * sizeof(float4);
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

// One step from buffer `start` and the bead-block read-out after it, as one
// graph; the read-out kernel's node (its destination is a placeholder, set
// before every launch) is kept with the graph it belongs to.
cudaError_t capture_read(lbmd_ctx *c, int start) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->own, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = enqueue_step(c, start);
  if (e2 == cudaSuccess) e2 = launch_bead_block(c->chain, c->status, c->stage, c->own);
  e = cudaStreamEndCapture(c->own, &g);
  if (e2 == cudaSuccess) e2 = e;
  size_t n = 0;
  if (e2 == cudaSuccess) e2 = cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (e2 == cudaSuccess && n > 0) e2 = cudaGraphGetNodes(g, nodes.data(), &n);
  cudaGraphNode_t found = nullptr;
  cudaKernelNodeParams kp = {};
  for (size_t k = 0; k < n && e2 == cudaSuccess && !found; ++k) {
    cudaGraphNodeType ty;
    if ((e2 = cudaGraphNodeGetType(nodes[k], &ty)) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams q = {};
    if ((e2 = cudaGraphKernelNodeGetParams(nodes[k], &q)) != cudaSuccess) break;
    if (q.func == bead_block_kernel()) {
      found = nodes[k];
      kp = q;
    }
  }
  if (e2 == cudaSuccess && !found) e2 = cudaErrorInvalidValue;
  cudaGraphExec_t ex = nullptr;
  if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority);
  if (e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e2;
  }
  c->rtmpl[start] = g;
  c->rgraph[start] = ex;
  c->rnode[start] = found;
  kp.kernelParams = nullptr;  // rebuilt per launch
  kp.extra = nullptr;
  c->rparams[start] = kp;
  return cudaSuccess;
}

// The chain's buffers (positions through the status word: ~1 MB for 400
// beads) as an L2-persisting window of the side stream, whose kernels (the MD
// cycle, the spread sums) run beside the stream-collide: its 637 MB per step
// would otherwise evict them from the 126 MB L2 between steps.  Raises the
// context's persisting-L2 limit to the window if it is lower.  Best effort:
// a device without persisting L2 keeps the default policy.  FP16 coupled step
// 85.4 -> 83.8 us on the 256x128x128, N = 400 box.
void keep_chain_in_l2(lbmd_ctx *c, const Layout &L) {
  const size_t bytes = (L.status + sizeof(DevStatus)) - L.pos;
  int dev = 0, max_window = 0;
  size_t limit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess ||
      max_window <= 0 || bytes > (size_t)max_window ||
      cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  if (limit < bytes && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  cudaStreamAttrValue v = {};
  v.accessPolicyWindow.base_ptr = c->ws + L.pos;
  v.accessPolicyWindow.num_bytes = bytes;
  v.accessPolicyWindow.hitRatio = 1.0f;
  v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  if (cudaStreamSetAttribute(c->side, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess)
    (void)cudaGetLastError();
}

void destroy_ctx(lbmd_ctx *c) {
  if (!c) return;
  for (auto &row : c->graph)
    for (auto &gx : row)
      if (gx) cudaGraphExecDestroy(gx);
  for (cudaGraphExec_t ex : c->tgraphs) cudaGraphExecDestroy(ex);
  for (int k = 0; k < 2; ++k) {
    if (c->rgraph[k]) cudaGraphExecDestroy(c->rgraph[k]);
    if (c->rtmpl[k]) cudaGraphDestroy(c->rtmpl[k]);
  }
  for (cudaEvent_t ev : c->tev) cudaEventDestroy(ev);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->own) cudaStreamDestroy(c->own);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->pinned) cudaFreeHost(c->pinned);
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

const char *lbmd_last_message(void) { return last_message(); }

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
  *bytes = make_layout(*params, true).total;
  return LBMD_OK;
}

int lbmd_create(const lbmd_params *params, void *dev_workspace, size_t bytes, void *cuda_stream,
                lbmd_ctx **out) {
  if (!out) return fail(LBMD_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  // without init_pos the chain starts from the library's seeded walk
  lbmd_params p = *params;
  std::vector<double> start;
  if (!p.init_pos && p.n_beads > 0) {
    if ((rc = seeded_start(p, start)) != LBMD_OK) return rc;
    p.init_pos = start.data();
  }
  Layout L = make_layout(p, true);
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
  c->aa = p.streaming == LBMD_STREAM_AA ? 1 : 0;
  c->user = (cudaStream_t)cuda_stream;
  c->N = p.n_beads;
  c->has_bonds = params_have_bonds(p) ? 1 : 0;
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

  if (c->N > 0) keep_chain_in_l2(c, L);
  Instance in;
  const char *what = "create";
  if ((e = init_instance(p, L, c->ws, c->user, in, &what)) != cudaSuccess) return bail(e, what);
  c->geo = in.geo;
  c->phys = in.phys;
  c->chain = in.chain;
  if (c->N > 0 &&
      cudaHostAlloc((void **)&c->pinned, bead_span(c) + sizeof(DevStatus), cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaGetLastError();  // no pinned staging: host read-outs copy pageable
    c->pinned = nullptr;
  }
  *out = c;
  return LBMD_OK;
}

int lbmd_step(lbmd_ctx *c, int64_t n_steps) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_steps < 0) return fail(LBMD_EINVAL, "n_steps < 0");
  if (n_steps == 0) return LBMD_OK;
  c->status_fresh = 0;
  if (c->timing) {
    // the n steps captured into one graph with event-record nodes around the
    // kernels (six events per step, reserved here), launched into the
    // caller's stream like the step graphs; kept until the times are read
    if (n_steps > (1 << 20)) return fail(LBMD_EINVAL, "at most 2^20 timed steps per call");
    const size_t need = c->tev_used + 6 * (size_t)n_steps;
    while (c->tev.size() < need) {
      cudaEvent_t ev;
      CK(c, cudaEventCreate(&ev));
      c->tev.push_back(ev);
    }
    cudaGraphExec_t ex = nullptr;
    CK(c, capture(c, c->cur, (int)n_steps, &ex));
    c->tgraphs.push_back(ex);
    CK(c, cudaGraphLaunch(ex, c->user));
    if (n_steps & 1) c->cur ^= 1;
    return LBMD_OK;
  }
  // graphs (captured on the private streams) launch straight into the
  // caller's stream: no cross-stream handshake per call
  int64_t left = n_steps;
  for (int gi = 2; gi >= 0; --gi) {
    const int len = kGraphSteps[gi];
    while (left >= len) {
      if (!c->graph[c->cur][gi]) CK(c, capture(c, c->cur, len, &c->graph[c->cur][gi]));
      CK(c, cudaGraphLaunch(c->graph[c->cur][gi], c->user));
      if (len & 1) c->cur ^= 1;
      left -= len;
    }
  }
  return LBMD_OK;
}

int lbmd_step_read_async(lbmd_ctx *c, void *dst, size_t bytes) {
  int rc = check_ctx(c);
  if (rc) return rc;
  const size_t need = kBeadBlockHeader + 48 * (size_t)c->N;
  if (!dst || bytes < need) return fail(LBMD_EINVAL, "dst is NULL or smaller than %zu bytes", need);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, dst) != cudaSuccess) {
    (void)cudaGetLastError();  // clear: the pointer is just not known to CUDA
    at.type = cudaMemoryTypeUnregistered;
    at.devicePointer = nullptr;
  }
  if (c->timing || at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) {
    // the two calls it stands for (timed steps, or memory the device cannot
    // address: the staged copy)
    if ((rc = lbmd_step(c, 1))) return rc;
    return lbmd_read_beads_async(c, dst, bytes);
  }
  const int k = c->cur;
  if (!c->rgraph[k]) CK(c, capture_read(c, k));
  const ChainArgs &a = c->chain;
  const float4 *pos = a.pos, *pos_lo = a.pos_lo, *vel = a.vel;
  int N = a.N, ox = a.ox, oy = a.oy, oz = a.oz;
  const DevStatus *st = c->status;
  char *out = (char *)at.devicePointer;
  void *args[9] = {&pos, &pos_lo, &vel, &N, &ox, &oy, &oz, &st, &out};
  cudaKernelNodeParams kp = c->rparams[k];
  kp.kernelParams = args;
  CK(c, cudaGraphExecKernelNodeSetParams(c->rgraph[k], c->rnode[k], &kp));
  CK(c, cudaGraphLaunch(c->rgraph[k], c->user));
  c->cur ^= 1;
  c->status_fresh = 0;
  return LBMD_OK;
}

int lbmd_read_fields(lbmd_ctx *c, float *rho, float *u, int dst_is_device) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!rho && !u) return LBMD_OK;
  const LbGeom &g = c->geo;
  const void *src = c->pop[c->cur];
  const int mode = pop_mode(c, c->cur);
  if (dst_is_device) {
    CK(c, launch_read_moments(c->p.storage, g, c->phys, src, mode, 0, g.nz, rho, u, g.V, c->user));
    return LBMD_OK;
  }
  const long long plane = (long long)g.nx * g.ny;
  const long long nzc_max = std::max(1LL, c->L.chunk_cells / plane);
  float *srho = c->stage, *su = c->stage + nzc_max * plane;
  for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
    const long long nzc = std::min(nzc_max, (long long)g.nz - z0);
    const long long cells = nzc * plane;
    CK(c, launch_read_moments(c->p.storage, g, c->phys, src, mode, z0, nzc, rho ? srho : nullptr,
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
  const int mode = pop_mode(c, c->cur);
  if (dst_is_device) {
    CK(c, launch_read_pulled(c->p.storage, g, (float)c->p.rho0, src, mode, 0, g.nz, f, g.V, c->user));
    return LBMD_OK;
  }
  const long long plane = (long long)g.nx * g.ny;
  const long long nzc_max = std::max(1LL, c->L.chunk_cells / plane);
  for (long long z0 = 0; z0 < g.nz; z0 += nzc_max) {
    const long long nzc = std::min(nzc_max, (long long)g.nz - z0);
    const long long cells = nzc * plane;
    CK(c, launch_read_pulled(c->p.storage, g, (float)c->p.rho0, src, mode, z0, nzc, c->stage, cells,
                             c->user));
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
  if (!dst_is_device && !aux && c->pinned) {
    // the position (hi, lo) and velocity arrays are adjacent in the workspace:
    // one copy of the span and one of the status word into pinned memory, one
    // synchronisation, then unwrapped x = origin + hi + lo in double on the host
    const size_t span = bead_span(c);
    CK(c, cudaMemcpyAsync(c->pinned, a.pos, span, cudaMemcpyDeviceToHost, c->user));
    CK(c, cudaMemcpyAsync(c->pinned + span, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                          c->user));
    CK(c, cudaStreamSynchronize(c->user));
    const float4 *hp = (const float4 *)c->pinned;
    const float4 *hl = (const float4 *)(c->pinned + (c->L.pos_lo - c->L.pos));
    const float4 *hv = (const float4 *)(c->pinned + (c->L.vel - c->L.pos));
    for (int i = 0; i < N; ++i) {
      if (x) {
        x[3 * i] = (double)a.ox + (double)hp[i].x + (double)hl[i].x;
        x[3 * i + 1] = (double)a.oy + (double)hp[i].y + (double)hl[i].y;
        x[3 * i + 2] = (double)a.oz + (double)hp[i].z + (double)hl[i].z;
      }
      if (y) {
        y[3 * i] = hv[i].x;
        y[3 * i + 1] = hv[i].y;
        y[3 * i + 2] = hv[i].z;
      }
    }
    memcpy(&c->status_cache, c->pinned + span, sizeof(DevStatus));
    c->status_fresh = 1;
    return LBMD_OK;
  }
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

int lbmd_read_beads_async(lbmd_ctx *c, void *dst, size_t bytes) {
  int rc = check_ctx(c);
  if (rc) return rc;
  const size_t need = kBeadBlockHeader + 48 * (size_t)c->N;
  if (!dst || bytes < need) return fail(LBMD_EINVAL, "dst is NULL or smaller than %zu bytes", need);
  // page-locked memory the device can address (cudaHostAlloc, or registered
  // as mapped): the kernel writes the block into it directly; otherwise it
  // fills the staging buffer and one copy moves it
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, dst) != cudaSuccess) {
    (void)cudaGetLastError();  // clear: the pointer is just not known to CUDA
    at.type = cudaMemoryTypeUnregistered;
    at.devicePointer = nullptr;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) {
    CK(c, launch_bead_block(c->chain, c->status, at.devicePointer, c->user));
    return LBMD_OK;
  }
  CK(c, launch_bead_block(c->chain, c->status, c->stage, c->user));
  CK(c, cudaMemcpyAsync(dst, c->stage, need, cudaMemcpyDeviceToHost, c->user));
  return LBMD_OK;
}

int lbmd_read_bead_aux(lbmd_ctx *c, double *u_i, double *impulse, int dst_is_device) {
  return read_bead_pair(c, u_i, impulse, dst_is_device, true);
}

int lbmd_status(lbmd_ctx *c, int64_t *step, int32_t *n_trans, int32_t *state, int64_t *t_transloc) {
  int rc = check_ctx(c);
  if (rc) return rc;
  DevStatus st;
  if (c->status_fresh) {
    st = c->status_cache;  // copied by the last host bead read-out, no step since
  } else {
    CK(c, cudaMemcpyAsync(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->user));
    CK(c, cudaStreamSynchronize(c->user));
  }
  if (step) *step = st.step;
  if (n_trans) *n_trans = st.n_trans;
  // a box without beads has no apply kernel to fold the population flag in
  if (state) *state = st.state == LBMD_RUNNING && st.pop_bad ? LBMD_NAN : st.state;
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
  CK(c, cudaStreamSynchronize(c->user));
  CK(c, cudaStreamSynchronize(c->own));
  for (cudaGraphExec_t ex : c->tgraphs) cudaGraphExecDestroy(ex);
  c->tgraphs.clear();
  c->timing = enable ? 1 : 0;
  c->tev_used = 0;
  c->timed_ms[0] = c->timed_ms[1] = c->timed_ms[2] = 0;
  c->timed_count = 0;
  return LBMD_OK;
}

static int collect_times(lbmd_ctx *c) {
  CK(c, cudaStreamSynchronize(c->user));
  CK(c, cudaStreamSynchronize(c->own));
  CK(c, cudaStreamSynchronize(c->side));
  for (cudaGraphExec_t ex : c->tgraphs) cudaGraphExecDestroy(ex);
  c->tgraphs.clear();
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

int lbmd_read_diagnostics(lbmd_ctx *c, lbmd_diag *records, int32_t max_records,
                          int32_t *n_records) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(c, cudaEventRecord(c->ev_in, c->own));
  CK(c, cudaStreamWaitEvent(c->user, c->ev_in, 0));
  return copy_diagnostics(c->status, c->chain.diag, c->p.diag_capacity, records, max_records,
                          n_records, c->user);
}

int lbmd_destroy(lbmd_ctx *c) {
  if (!c) return LBMD_OK;
  cudaStreamSynchronize(c->user);
  cudaStreamSynchronize(c->own);
  cudaStreamSynchronize(c->side);
  destroy_ctx(c);
  return LBMD_OK;
}

}  // extern "C"

