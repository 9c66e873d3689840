// libdiffrestore C ABI: context, device memory, scene upload and the host
// orchestration of Alg. 1 - 3 (see include/diffrestore.h for the contract).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "../../include/diffrestore.h"
#include "dr_internal.h"

using namespace dr;

namespace {
float hbits_f(int v) { float f; std::memcpy(&f, &v, 4); return f; }

// Runs f(begin, end, part) over [0, n) in up to 16 contiguous parts on host
// threads (one part below 2^16 items); parts are numbered in order, so
// per-part results joined in part order are those of one sequential pass.
template <class F>
int parallel_parts(long long n, F f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int parts = n < (1ll << 16) ? 1 : (int)std::min<unsigned>(16u, hw);
  if (parts == 1) {
    f(0ll, n, 0);
    return 1;
  }
  std::vector<std::thread> th;
  for (int p = 0; p < parts; ++p) {
    try {
      th.emplace_back(f, n * p / parts, n * (p + 1) / parts, p);
    } catch (...) {  // no thread to be had: this part on the calling thread
      f(n * p / parts, n * (p + 1) / parts, p);
    }
  }
  for (auto& t : th) t.join();
  return parts;
}

// Runs f(i) for i in [0, n) on up to 16 host threads taking items one at a
// time (for few, unequal items); f must write disjoint outputs.
template <class F>
void parallel_items(int n, F f) {
  const int nth = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) f(i);
  };
  if (nth == 1 || n < 2) {
    work();
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < std::min(nth, n); ++t) {
    try {
      th.emplace_back(work);
    } catch (...) {  // fewer threads: the others and the caller finish the items
      break;
    }
  }
  work();
  for (auto& t : th) t.join();
}
int hbits_i(float f) { int v; std::memcpy(&v, &f, 4); return v; }
}  // namespace

struct dr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // target
  int target = -1;  // -1 none, 0 scene, 1 mixture
  int W = 0, H = 0;
  int nt = 0, n_nodes = 0, n_lights = 0;
  float tmin = 0.f;
  Camera cam{};
  float4* nodes = nullptr;
  float4* tris = nullptr;
  float4* nodes4 = nullptr;  // 4-wide collapse of `nodes` (null when not built)
  float4* tris4 = nullptr;
  int n_nodes4 = 0, bvh4_depth = 0, bvh4_stack = 0;
  double bvh4_sah_nodes = 0.0, bvh4_sah_tris = 0.0;  // SAH cost terms of the 4-wide BVH
  uint4* nodes8 = nullptr;  // 8-wide compressed collapse (built when bvh_width is 8 at upload)
  float4* tris8 = nullptr;
  int n_nodes8 = 0, bvh8_depth = 0;
  bool batch_bvh8 = false;  // every scene of the batch has an 8-wide BVH
  // two-level BVH of an instanced scene (null: none)
  float4* tl_nodes = nullptr;
  float4* bl_nodes = nullptr;
  float4* bl_tris = nullptr;
  float4* insts = nullptr;
  int n_tl_nodes = 0, n_bl_nodes = 0, n_bl_tris = 0, n_insts = 0;
  int two_level = 0;  // DR_OPT_TWO_LEVEL
  int bvh_width = 0;  // DR_OPT_BVH_WIDTH (0 automatic)
  bool conductors = false;  // some material is a conductor (selects the kernels that shade them)
  unsigned long long target_gen = 0;  // bumped by every scene / mixture upload
  // multi-scene batch (target 2): one sub-context per scene owns that
  // scene's BVH and surface data; the kernels see them through d_scenes
  std::vector<dr_ctx*> subs;
  std::vector<SceneChains> h_sc;   // per scene: chain range, L, d, first pixel, k0, tour counter
  std::vector<int> batch_w, batch_h;
  DevScene* d_scenes = nullptr;
  SceneChains* d_sc = nullptr;
  uint8_t* chain_scene = nullptr;  // [N]
  unsigned long long* batch_tours = nullptr;  // [n_scenes]
  double* batch_psum = nullptr;               // [n_scenes]
  WfTuning tune;                              // DR_OPT_TRAVERSE_BLOCKS, DR_OPT_REFILL
  int ray_order = -1;                         // DR_OPT_RAY_ORDER (-1 automatic)
  int tail_bounce = -1;                       // DR_OPT_TAIL_BOUNCE (-1 automatic)
  float4* surf = nullptr;
  float4* lights = nullptr;
  float* nrm = nullptr;
  float* mats = nullptr;
  float* mw = nullptr;
  float* mmu = nullptr;
  float* msig = nullptr;
  int mK = 0, md = 0;
  float mcval = 0.f;
  // chains
  unsigned long long N = 0;
  int d = 0;
  dr_params prm{};
  uint32_t step = 0;
  uint64_t seed = 0;
  uint32_t frame = 0;
  bool inited = false;
  float* x = nullptr;
  float* score = nullptr;
  float* xp = nullptr;     // MALA: proposal [d][N]
  float* sp = nullptr;     // MALA: score at the proposal [d][N]
  float4* cur = nullptr;   // MALA: f and pixel of the current state [N]
  size_t mala_cap = 0;     // chains * d the MALA buffers hold
  float* logp = nullptr;
  uint8_t* killed = nullptr;
  uint8_t* plen = nullptr;      // [N] last path length (work-order key)
  uint2* order_a = nullptr;     // [N] (key, chain) pairs and the sort's ping-pong buffer
  uint2* order_b = nullptr;
  SplatRec* rec = nullptr;
  SplatRec* rec_alt = nullptr;
  size_t rec_cap = 0;  // steps
  uint32_t rec_count = 0;
  void* sort_scratch = nullptr;
  size_t state_cap = 0;  // N * d allocated
  size_t chains_cap = 0;
  size_t rec_cap_records = 0;
  double* accum = nullptr;
  size_t accum_n = 0;
  unsigned long long* counters = nullptr;  // tour_count, rays, node visits, tri tests
  double* p_partial = nullptr;
  size_t p_partial_cap = 0;
  double* p_sum = nullptr;
  uint32_t* err = nullptr;
  unsigned long long launches = 0;  // kernels launched by this context
  double k0 = 0.0;
  double p_lambda = 0.0;
  double p_init_sum = 0.0;          // sum of p over the initial samples of the last estimate
  unsigned long long p_init_n = 0;  // their count (0: no estimate)
  bool stats = false;
  int builder = DR_BVH_PLOC;
  int ploc_radius = 16;
  int work_order = 0;  // DR_OPT_WORK_ORDER
  int wavefront = -1;  // DR_OPT_WAVEFRONT: -1 auto (N >= 2^17), 0 fused, 1 wavefront
  void* wf_mem = nullptr;
  size_t wf_cap = 0;
  int n_sm = 152;
  // graph-captured frames (dr_frame)
  FrameParams* frame_dev = nullptr;  // what a replayed frame graph reads (step, RNG key, k0)
  bool capturing = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned long long> graph_key;  // what the captured launches depend on
  unsigned long long graph_launches = 0;
  FrameParams frame_host{};  // source of the per-launch copy into frame_dev
  // optional per-phase timing (DR_OPT_PROFILE)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Mark {
    int phase, bounce;
    cudaEvent_t begin, end;
  };
  std::vector<Mark> marks;
  cudaEvent_t open_ev[kPhCount] = {};
  double phase_ms[kPhCount] = {};
  unsigned long long phase_n[kPhCount] = {};
  double bounce_ms[3][kMaxPathLen + 1] = {};  // trace, shade, shadow per bounce
  unsigned long long bounce_rays[2][kMaxPathLen + 1] = {};  // closest-hit, shadow rays per bounce
};

namespace {

cudaEvent_t pooled_event(dr_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records an event at the start / end of a phase on the context's stream.
void phase_mark(void* user, int phase, bool begin, int bounce) {
  dr_ctx* c = static_cast<dr_ctx*>(user);
  if (!c->profile || c->capturing) return;
  cudaEvent_t e = pooled_event(c);
  if (!e) return;
  cudaEventRecord(e, c->stream);
  if (begin) {
    c->open_ev[phase] = e;
  } else if (c->open_ev[phase]) {
    c->marks.push_back({phase, bounce, c->open_ev[phase], e});
    c->open_ev[phase] = nullptr;
  } else {
    c->ev_pool.push_back(e);
  }
}

// Folds finished event pairs into the per-phase totals (synchronises).
void phase_collect(dr_ctx* c) {
  if (c->marks.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& m : c->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.begin, m.end) == cudaSuccess) {
      c->phase_ms[m.phase] += ms;
      c->phase_n[m.phase] += 1;
      const int row = m.phase == kPhTrace ? 0 : m.phase == kPhShade ? 1 : m.phase == kPhShadow ? 2 : -1;
      if (row >= 0 && m.bounce >= 1 && m.bounce <= kMaxPathLen) c->bounce_ms[row][m.bounce] += ms;
    }
    c->ev_pool.push_back(m.begin);
    c->ev_pool.push_back(m.end);
  }
  cudaGetLastError();
  c->marks.clear();
}

}  // namespace

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

void dr::set_error_message(const char* msg) { g_err = msg; }

namespace {

#define DR_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? DR_ERR_OOM : DR_ERR_CUDA,                      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    }                                                                                              \
  } while (0)

template <class T>
int dalloc(T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) return DR_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(DR_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes: " +
                                cudaGetErrorString(e));
  }
  return DR_OK;
}

template <class T>
void dfree(T** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

#define DR_TRY(expr)             \
  do {                           \
    int r_ = (expr);             \
    if (r_ != DR_OK) return r_;  \
  } while (0)

// Kernel view of the uploaded scene: the 4-wide BVH unless the binary one
// is asked for (DR_OPT_BVH_WIDTH = 2) or none was built.
DevScene dev_scene(const dr_ctx* c) {
  DevScene S;
  S.nodes = c->nodes;
  S.tris = c->tris;
  S.surf = c->surf;
  S.nrm = c->nrm;
  S.mats = c->mats;
  S.lights = c->lights;
  S.n_lights = c->n_lights;
  S.n_tris = c->nt;
  S.n_nodes = std::max(1, c->n_nodes);
  const bool wide = c->nodes4 != nullptr && c->bvh_width != 2;
  S.nodes4 = wide ? c->nodes4 : nullptr;
  S.tris4 = wide ? c->tris4 : nullptr;
  S.n_nodes4 = wide ? c->n_nodes4 : 0;
  const bool tl = c->tl_nodes != nullptr && c->two_level != 0;
  S.tl_nodes = tl ? c->tl_nodes : nullptr;
  S.bl_nodes = tl ? c->bl_nodes : nullptr;
  S.bl_tris = tl ? c->bl_tris : nullptr;
  S.insts = tl ? c->insts : nullptr;
  S.n_tl_nodes = tl ? c->n_tl_nodes : 0;
  S.n_bl_nodes = tl ? c->n_bl_nodes : 0;
  S.n_bl_tris = tl ? c->n_bl_tris : 0;
  S.n_insts = tl ? c->n_insts : 0;
  const bool w8 = wide && c->nodes8 != nullptr && c->bvh_width == 8;
  S.nodes8 = w8 ? c->nodes8 : nullptr;
  S.tris8 = w8 ? c->tris8 : nullptr;
  S.n_nodes8 = w8 ? c->n_nodes8 : 0;
  S.W = c->W;
  S.H = c->H;
  S.tmin = c->tmin;
  S.cam = c->cam;
  return S;
}

DevMixture dev_mixture(const dr_ctx* c) {
  DevMixture M;
  M.w = c->mw;
  M.mu = c->mmu;
  M.sig = c->msig;
  M.K = c->mK;
  M.d = c->md;
  M.W = c->W;
  M.H = c->H;
  M.cval = c->mcval;
  return M;
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return DR_OK;
}

int key_bits(long long n_pix) {
  int b = 0;
  while (b < 32 && (1ll << b) < n_pix) ++b;
  return std::max(b, 1);
}

int check_device_error(dr_ctx* c) {
  uint32_t e = 0;
  DR_CUDA(cudaMemcpyAsync(&e, c->err, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  if (e) {
    std::string m = "device check failed:";
    if (e & kErrStackOverflow) m += " traversal stack overflow;";
    if (e & kErrNonFinite) m += " non-finite f or p;";
    if (e & kErrBadIndex) m += " index out of range;";
    if (e & kErrTimeout) m += " bounded wait timed out;";
    return fail(e & kErrTimeout ? DR_ERR_TIMEOUT : DR_ERR_DEVICE_CHECK, m);
  }
  return DR_OK;
}

int flush(dr_ctx* c) {
  if (c->rec_count == 0) return DR_OK;
  const size_t n = (size_t)c->rec_count * c->N;
  phase_mark(c, kPhSplat, true, 0);
  SplatRec* sorted =
      sort_splat_records(c->rec, c->rec_alt, n, key_bits((long long)c->W * c->H), c->sort_scratch, c->stream);
  launch_segment_reduce(sorted, n, c->accum, (uint32_t)((size_t)c->W * c->H), c->err, c->stream);
  phase_mark(c, kPhSplat, false, 0);
  c->launches += 5 * ((key_bits((long long)c->W * c->H) + 7) / 8) + 1;
  c->rec_count = 0;
  return check_launch("splat");
}

bool use_wavefront(const dr_ctx* c);

StepArgs step_args(dr_ctx* c) {
  StepArgs a{};
  a.S = dev_scene(c);
  a.M = dev_mixture(c);
  a.target = c->target;
  a.x = c->x;
  a.score = c->score;
  a.xp = c->xp;
  a.sp = c->sp;
  a.cur = c->cur;
  a.killed = c->killed;
  a.logp = c->logp;
  a.N = c->N;
  a.d = c->d;
  a.L = c->prm.max_path_len;
  a.rng = Rng{(uint32_t)c->seed, (uint32_t)(c->seed >> 32), c->frame};
  a.stddev = c->prm.stddev;
  a.gamma_tilde = c->prm.gamma_tilde;
  a.h = 1.0f / c->prm.dt;
  a.eps = c->prm.eps;
  a.k0 = c->k0;
  a.rb = c->prm.rb_weight;
  a.drift = c->prm.drift_mode;
  a.tour_count = c->counters + 0;
  a.rays = c->counters + 1;
  a.node_visits = c->counters + 2;
  a.tri_tests = c->counters + 3;
  a.err = c->err;
  a.refill = c->tune.refill;
  a.conductors = c->conductors ? 1 : 0;
  a.bvh8 = c->target == 2 ? (c->batch_bvh8 && c->bvh_width == 8 ? 1 : 0) : (a.S.nodes8 != nullptr ? 1 : 0);
  a.two_level = c->target == 0 && a.S.tl_nodes != nullptr ? 1 : 0;
  if (c->target == 2) {
    a.scenes = c->d_scenes;
    a.sc = c->d_sc;
    a.chain_scene = c->chain_scene;
    a.target = 0;
  }
  return a;
}

int run_fd(dr_ctx* c) {
  FdArgs f{};
  f.S = dev_scene(c);
  f.M = dev_mixture(c);
  f.target = c->target;
  f.x = c->x;
  f.score = c->score;
  f.killed = c->killed;
  f.N = c->N;
  f.d = c->d;
  f.L = c->prm.max_path_len;
  f.eps = c->prm.eps;
  f.fd_h = c->prm.fd_h;
  f.rays = c->counters + 1;
  f.err = c->err;
  launch_fd_score(f, c->stream);
  c->launches += 1;
  return check_launch("fd_score");
}

bool use_wavefront(const dr_ctx* c) {
  if (c->target == 2) return true;  // a batch runs bounce by bounce only
  // the bounce-by-bounce passes compute the adjoint drift, or no drift
  const bool wf_drift = c->prm.drift_mode == DR_DRIFT_ADJOINT || c->prm.drift_mode == DR_DRIFT_NONE;
  return wf_drift && c->target == 0 && (c->wavefront == 1 || (c->wavefront == -1 && c->N >= (1ull << 17)));
}

int ensure_wavefront_buffers(dr_ctx* c) {
  const size_t need = wf_bytes(c->N, c->prm.max_path_len);
  if (need <= c->wf_cap) return DR_OK;
  if (c->wf_mem) cudaFree(c->wf_mem);
  c->wf_mem = nullptr;
  c->wf_cap = 0;
  cudaError_t e = cudaMalloc(&c->wf_mem, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->wf_mem = nullptr;
    return fail(DR_ERR_OOM, "wavefront buffers");
  }
  c->wf_cap = need;
  return DR_OK;
}

// one chain step (init = Alg. 1, else Alg. 2); records into the next slot
// Camera-ray ordering for the bounce-by-bounce passes (DR_OPT_RAY_ORDER):
// Morton keys over the largest image side, above them the scene index of a
// batch; off when the key would not fit 32 bits.
RayOrder ray_order(dr_ctx* c, StepArgs& a) {
  RayOrder o;
  // automatic: on for large geometry, where coherent camera rays save more
  // traversal time than the sort and the scattered slot accesses cost
  // (measured: +5% at 1M triangles, +7% for a 2M-triangle batch, -5% at 20k)
  const bool on = c->ray_order == 1 || (c->ray_order == -1 && c->nt >= (1 << 17));
  if (!on || !c->order_a || !c->order_b || !c->sort_scratch) return o;
  int side = c->target == 2 ? 1 : std::max(c->W, c->H);
  for (size_t q = 0; q < c->batch_w.size(); ++q) side = std::max(side, std::max(c->batch_w[q], c->batch_h[q]));
  int b = 0;
  while ((1 << b) < side) ++b;
  int sb = 0;
  while ((1u << sb) < (unsigned)std::max<size_t>(1, c->h_sc.size())) ++sb;
  if (b > 16 || 2 * b + (c->target == 2 ? sb : 0) > 32) return o;
  o.keys = c->order_a;
  o.alt = c->order_b;
  o.scratch = c->sort_scratch;
  o.bits = 2 * b + (c->target == 2 ? sb : 0);
  a.key_shift = 2 * b;
  return o;
}

// The bounce from whose shading on a step runs as one persistent pass
// (DR_OPT_TAIL_BOUNCE; 0 none).  Automatic: from bounce 4 when paths reach
// 14 segments or more, where the late bounces hold few rays each (measured:
// +7% on the 64-scene batch with L up to 16; no gain at L = 12).
int tail_bounce(const dr_ctx* c) {
  if (c->tail_bounce >= 0) return c->tail_bounce;
  return c->prm.max_path_len >= 14 ? 4 : 0;
}

int one_step(dr_ctx* c, bool init) {
  if (!init && c->rec_count >= c->rec_cap) DR_TRY(flush(c));
  StepArgs a = step_args(c);
  a.init = init ? 1 : 0;
  a.step = c->step;
  a.fp = c->capturing ? c->frame_dev : nullptr;
  a.rec = c->rec + (size_t)c->rec_count * c->N;
  a.p_partial = init ? c->p_partial : nullptr;
  a.plen = c->plen;
  const PhaseHook hook{phase_mark, c};
  if (use_wavefront(c)) {
    DR_TRY(ensure_wavefront_buffers(c));
    const WfBuffers w = wf_carve(c->wf_mem, c->N, c->prm.max_path_len);
    const RayOrder ord = ray_order(c, a);
    WfTuning tune = c->tune;
    tune.tail_bounce = tail_bounce(c);
    c->launches += launch_wavefront_step(a, w, c->stats, c->n_sm, tune, hook, c->stream, kWfStep, nullptr, ord);
    DR_TRY(check_launch("wavefront step"));
    if (c->profile && !c->capturing) {
      // rays per bounce for the profile (profiling only: waits for the step)
      uint32_t n[kWfCounts];
      DR_CUDA(cudaMemcpyAsync(n, w.counts, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
      DR_CUDA(cudaStreamSynchronize(c->stream));
      for (int k = 1; k <= c->prm.max_path_len; ++k) {
        c->bounce_rays[0][k] += n[k];
        c->bounce_rays[1][k] += n[kWfShadowCount0 + k];
      }
    }
  } else {
    if (!init && c->work_order && c->prm.drift_mode == DR_DRIFT_ADJOINT && c->target == 0) {
      hook(kPhOrder, true);
      launch_order_keys(c->killed, c->plen, c->N, c->order_a, c->stream);
      a.order = sort_pairs(c->order_a, c->order_b, c->N, 6, c->sort_scratch, c->stream);
      hook(kPhOrder, false);
      c->launches += 6;
    }
    hook(kPhFused, true);
    launch_step(a, c->stats, c->stream);
    hook(kPhFused, false);
    c->launches += 1;
    DR_TRY(check_launch("restore_step"));
    if (c->prm.drift_mode == DR_DRIFT_FD) {
      hook(kPhFd, true);
      DR_TRY(run_fd(c));
      hook(kPhFd, false);
    }
  }
  c->rec_count++;
  if (c->capturing) {
    launch_advance_step(&c->frame_dev->step, c->stream);
    c->launches += 1;
  }
  return DR_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

// Releases a multi-scene batch (its per-scene contexts and tables).
void free_batch(dr_ctx* c) {
  for (dr_ctx* s : c->subs) dr_destroy(s);
  c->subs.clear();
  c->h_sc.clear();
  c->batch_w.clear();
  c->batch_h.clear();
  dfree(&c->d_scenes);
  dfree(&c->d_sc);
  dfree(&c->chain_scene);
  dfree(&c->batch_tours);
  dfree(&c->batch_psum);
}

// Checks the freshly built binary BVH on the device (a tree: every inner
// node but the root and every triangle referenced exactly once; its height
// to *depth2) and collapses it into the 4-wide layout.  Scenes of one
// triangle (whose binary tree repeats its leaf) are trivially fine and keep
// the binary BVH only, as do trees whose 4-wide traversal could need more
// stack than the kernels hold.
int build_bvh4(dr_ctx* c, int* depth2) {
  dfree(&c->nodes4);
  dfree(&c->tris4);
  c->n_nodes4 = c->bvh4_depth = c->bvh4_stack = 0;
  *depth2 = 1;
  if (c->nt < 2) return DR_OK;
  const int nn = std::max(1, c->n_nodes);
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, bvh4_scratch_bytes(nn, c->nt)) != cudaSuccess) {
    cudaGetLastError();
    return fail(DR_ERR_OOM, "dr_scene_upload: 4-wide BVH scratch");
  }
  Bvh4Plan plan{};
  int r = DR_OK;
  const int n4 = bvh4_plan(c->nodes, nn, c->nt, scratch, &plan, c->stream);
  c->launches += plan.launches;
  if (!plan.tree_ok) {
    r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload: the BVH is not a tree over the triangles");
  } else if (n4 >= 1) {
    *depth2 = plan.depth2;
    if (plan.stack_need <= kTraversalStack) {
      r = dalloc(&c->nodes4, (size_t)kNode4F4 * n4);
      if (r == DR_OK) r = dalloc(&c->tris4, (size_t)kTriF4 * c->nt);
      if (r == DR_OK && bvh4_emit(c->nodes, c->tris, nn, c->nt, scratch, c->nodes4, c->tris4, c->stream) < 0)
        r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload: 4-wide BVH emission failed");
      c->launches += 1;
      if (r == DR_OK) {
        c->n_nodes4 = n4;
        c->bvh4_depth = plan.depth;
        c->bvh4_stack = plan.stack_need;
        if (bvh4_sah(c->nodes4, n4, c->stream, &c->bvh4_sah_nodes, &c->bvh4_sah_tris) < 0)
          r = fail(DR_ERR_CUDA, "dr_scene_upload: SAH cost of the 4-wide BVH");
        c->launches += 5;
      } else {
        dfree(&c->nodes4);
        dfree(&c->tris4);
      }
    }
  } else {
    r = fail(DR_ERR_CUDA, "dr_scene_upload: BVH check / collapse failed");
  }
  cudaFree(scratch);
  const cudaError_t e = cudaGetLastError();
  if (r == DR_OK && e != cudaSuccess) r = fail(DR_ERR_CUDA, std::string("dr_scene_upload: ") + cudaGetErrorString(e));
  return r;
}

// The 8-wide compressed collapse (when the context asks for width 8 and the
// 4-wide one was built); kept off when its traversal could need more stack
// entries (two ints each) than the kernels hold.
int build_bvh8(dr_ctx* c) {
  dfree(&c->nodes8);
  dfree(&c->tris8);
  c->n_nodes8 = c->bvh8_depth = 0;
  if (c->bvh_width != 8 || !c->nodes4 || c->nt < 2) return DR_OK;
  const int nn = std::max(1, c->n_nodes);
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, bvh8_scratch_bytes(nn, c->nt)) != cudaSuccess) {
    cudaGetLastError();
    return fail(DR_ERR_OOM, "dr_scene_upload: 8-wide BVH scratch");
  }
  Bvh8Plan plan{};
  int r = DR_OK;
  const int n8 = bvh8_plan(c->nodes, nn, c->nt, scratch, &plan, c->stream);
  c->launches += plan.launches;
  if (n8 < 1) {
    r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload: 8-wide BVH collapse failed");
  } else if (plan.depth <= kTraversalStack / 2) {
    r = dalloc(&c->nodes8, (size_t)kNode8U4 * n8);
    if (r == DR_OK) r = dalloc(&c->tris8, (size_t)kTriF4 * c->nt);
    if (r == DR_OK && bvh8_emit(c->nodes, c->tris, nn, c->nt, scratch, n8, c->nodes8, c->tris8, c->stream) < 0)
      r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload: 8-wide BVH emission failed");
    c->launches += 2;
    if (r == DR_OK) {
      c->n_nodes8 = n8;
      c->bvh8_depth = plan.depth;
    } else {
      dfree(&c->nodes8);
      dfree(&c->tris8);
    }
  }
  cudaFree(scratch);
  const cudaError_t e = cudaGetLastError();
  if (r == DR_OK && e != cudaSuccess) r = fail(DR_ERR_CUDA, std::string("dr_scene_upload: ") + cudaGetErrorString(e));
  return r;
}

void free_two_level(dr_ctx* c) {
  dfree(&c->tl_nodes);
  dfree(&c->bl_nodes);
  dfree(&c->bl_tris);
  dfree(&c->insts);
  c->n_tl_nodes = c->n_bl_nodes = c->n_bl_tris = c->n_insts = 0;
}

// A 4-wide BVH over nt >= 2 triangles given on the host (binary build with
// the context's builder, then the collapse with leaves of at most
// max_leaf): *nodes4 [*n4 * 7] and *tris4 [nt * 3] (record id = triangle
// index in the input), allocated here.
int build_wide(dr_ctx* c, const float* verts, int nv, const int* tris, int nt, int max_leaf, float4** nodes4,
               float4** tris4, int* n4, int* stack_need) {
  cudaStream_t s = c->stream;
  float* dv = nullptr;
  int* dt = nullptr;
  float4 *n2 = nullptr, *t2 = nullptr;
  void *scratch = nullptr, *ploc = nullptr, *s4 = nullptr;
  int r = dalloc(&dv, 3 * (size_t)nv);
  if (r == DR_OK) r = dalloc(&dt, 3 * (size_t)nt);
  if (r == DR_OK) r = dalloc(&n2, 4 * (size_t)(nt - 1));
  if (r == DR_OK) r = dalloc(&t2, 3 * (size_t)nt);
  if (r == DR_OK) {
    cudaError_t e = cudaMalloc(&scratch, bvh_scratch_bytes(nt));
    if (e == cudaSuccess && c->builder == DR_BVH_PLOC) e = cudaMalloc(&ploc, ploc_scratch_bytes(nt));
    if (e == cudaSuccess) e = cudaMalloc(&s4, bvh4_scratch_bytes(nt - 1, nt));
    if (e != cudaSuccess) {
      cudaGetLastError();
      r = fail(DR_ERR_OOM, "dr_scene_upload_instanced: BVH scratch");
    }
  }
  if (r == DR_OK) {
    cudaMemcpyAsync(dv, verts, 12 * (size_t)nv, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dt, tris, 12 * (size_t)nt, cudaMemcpyHostToDevice, s);
    const int nn = c->builder == DR_BVH_PLOC ? build_ploc(dv, dt, nt, n2, t2, scratch, ploc, c->ploc_radius, kTraversalStack + 1, s)
                                             : build_lbvh(dv, dt, nt, n2, t2, scratch, s);
    c->launches += 8;
    Bvh4Plan plan{};
    const int m = nn < 1 ? -1 : bvh4_plan(n2, nn, nt, s4, &plan, s, max_leaf);
    c->launches += plan.launches;
    if (m < 1) {
      r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload_instanced: BLAS / TLAS construction failed");
    } else {
      r = dalloc(nodes4, (size_t)kNode4F4 * m);
      if (r == DR_OK) r = dalloc(tris4, (size_t)kTriF4 * nt);
      if (r == DR_OK && bvh4_emit(n2, t2, nn, nt, s4, *nodes4, *tris4, s) < 0)
        r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload_instanced: BLAS / TLAS emission failed");
      c->launches += 1;
      *n4 = m;
      *stack_need = plan.stack_need;
    }
  }
  dfree(&dv);
  dfree(&dt);
  dfree(&n2);
  dfree(&t2);
  if (scratch) cudaFree(scratch);
  if (ploc) cudaFree(ploc);
  if (s4) cudaFree(s4);
  if (r != DR_OK) {
    dfree(nodes4);
    dfree(tris4);
  }
  return r;
}

// The two-level BVH: BLAS per mesh (concatenated), TLAS over the instance
// boxes, instance records.  Left off (DR_OK, nothing built) when its walk
// could need more stack than the kernels hold.
int build_two_level(dr_ctx* c, const dr_mesh_desc* meshes, int nmesh, const dr_instance_desc* inst, int ninst,
                    const std::vector<double>& inv, const std::vector<int>& tri_base, const std::vector<float>& box) {
  free_two_level(c);
  cudaStream_t s = c->stream;
  std::vector<float4*> mn(nmesh, nullptr), mt(nmesh, nullptr);
  std::vector<int> n4(nmesh, 0), node_off(nmesh, 0), tri_off(nmesh, 0);
  int r = DR_OK, total_nodes = 0, total_tris = 0, blas_need = 0;
  for (int m = 0; m < nmesh && r == DR_OK; ++m) {
    const dr_mesh_desc& q = meshes[m];
    node_off[m] = total_nodes;
    tri_off[m] = total_tris;
    if (q.nt == 1) {
      // one triangle: a root with one leaf child
      const float* v0 = q.verts + 3 * q.tris[0];
      const float* v1 = q.verts + 3 * q.tris[1];
      const float* v2 = q.verts + 3 * q.tris[2];
      float lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(v0[a], std::min(v1[a], v2[a]));
        hi[a] = std::max(v0[a], std::max(v1[a], v2[a]));
      }
      float4 nd[kNode4F4];
      const float inf = std::numeric_limits<float>::infinity();
      for (int a = 0; a < 3; ++a) {
        // empty slots: inverted boxes, which no ray enters
        nd[2 * a] = make_float4(lo[a], inf, inf, inf);
        nd[2 * a + 1] = make_float4(hi[a], -inf, -inf, -inf);
      }
      nd[6] = make_float4(hbits_f(leaf_code(0, 1)), hbits_f(kBvh4Empty), hbits_f(kBvh4Empty), hbits_f(kBvh4Empty));
      const float4 tr[3] = {make_float4(v0[0], v0[1], v0[2], hbits_f(0)),
                            make_float4(v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2], 0.f),
                            make_float4(v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2], 0.f)};
      r = dalloc(&mn[m], kNode4F4);
      if (r == DR_OK) r = dalloc(&mt[m], 3);
      if (r == DR_OK) {
        cudaMemcpyAsync(mn[m], nd, sizeof(nd), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(mt[m], tr, sizeof(tr), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
      }
      n4[m] = 1;
    } else {
      int need = 0;
      r = build_wide(c, q.verts, q.nv, q.tris, q.nt, kBvh4MaxLeaf, &mn[m], &mt[m], &n4[m], &need);
      blas_need = std::max(blas_need, need);
    }
    total_nodes += n4[m];
    total_tris += q.nt;
  }
  if (r == DR_OK) r = dalloc(&c->bl_nodes, (size_t)kNode4F4 * total_nodes);
  if (r == DR_OK) r = dalloc(&c->bl_tris, (size_t)kTriF4 * total_tris);
  for (int m = 0; m < nmesh && r == DR_OK; ++m) {
    cudaMemcpyAsync(c->bl_nodes + (size_t)kNode4F4 * node_off[m], mn[m], 16 * (size_t)kNode4F4 * n4[m],
                    cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->bl_tris + (size_t)kTriF4 * tri_off[m], mt[m], 16 * (size_t)kTriF4 * meshes[m].nt,
                    cudaMemcpyDeviceToDevice, s);
    launch_link_offset(c->bl_nodes + (size_t)kNode4F4 * node_off[m], n4[m], node_off[m], tri_off[m], s);
    c->launches += 1;
  }
  if (r == DR_OK) cudaStreamSynchronize(s);
  for (int m = 0; m < nmesh; ++m) {
    dfree(&mn[m]);
    dfree(&mt[m]);
  }
  // TLAS over the instance boxes, each given as the degenerate triangle
  // (lo, hi, lo) whose box it is
  float4* tl_tris = nullptr;
  int tl_need = 0;
  if (r == DR_OK) {
    std::vector<float> bv(9 * (size_t)ninst);
    std::vector<int> bt(3 * (size_t)ninst);
    for (int i = 0; i < ninst; ++i) {
      for (int a = 0; a < 3; ++a) {
        bv[9 * i + a] = box[6 * i + a];
        bv[9 * i + 3 + a] = box[6 * i + 3 + a];
        bv[9 * i + 6 + a] = box[6 * i + a];
      }
      for (int k = 0; k < 3; ++k) bt[3 * i + k] = 3 * i + k;
    }
    r = build_wide(c, bv.data(), 3 * ninst, bt.data(), ninst, 1, &c->tl_nodes, &tl_tris, &c->n_tl_nodes, &tl_need);
  }
  uint32_t* derr = nullptr;
  if (r == DR_OK) r = dalloc(&derr, 1);
  if (r == DR_OK) {
    cudaMemsetAsync(derr, 0, 4, s);
    launch_tlas_leaves(c->tl_nodes, c->n_tl_nodes, tl_tris, ninst, derr, s);
    c->launches += 1;
    uint32_t e = 0;
    cudaMemcpyAsync(&e, derr, 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || e != 0)
      r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload_instanced: TLAS leaves");
  }
  dfree(&derr);
  dfree(&tl_tris);
  // instance records
  if (r == DR_OK) {
    std::vector<float4> ir(kInstF4 * (size_t)ninst);
    for (int i = 0; i < ninst; ++i) {
      const double* M = inv.data() + 12 * (size_t)i;
      for (int row = 0; row < 3; ++row)
        ir[kInstF4 * i + row] = make_float4((float)M[4 * row], (float)M[4 * row + 1], (float)M[4 * row + 2],
                                            (float)M[4 * row + 3]);
      ir[kInstF4 * i + 3] = make_float4(hbits_f(node_off[inst[i].mesh]), hbits_f(tri_base[i]), 0.f, 0.f);
    }
    r = dalloc(&c->insts, ir.size());
    if (r == DR_OK) {
      cudaMemcpyAsync(c->insts, ir.data(), 16 * ir.size(), cudaMemcpyHostToDevice, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) r = fail(DR_ERR_CUDA, "dr_scene_upload_instanced: copy");
    }
  }
  if (r == DR_OK) {
    c->n_bl_nodes = total_nodes;
    c->n_bl_tris = total_tris;
    c->n_insts = ninst;
    // the walk holds the TLAS path, one return mark and a BLAS path
    if (tl_need + 1 + blas_need > kTraversalStackTL) free_two_level(c);
  } else {
    free_two_level(c);
  }
  const cudaError_t e = cudaGetLastError();
  if (r == DR_OK && e != cudaSuccess) r = fail(DR_ERR_CUDA, std::string("dr_scene_upload_instanced: ") + cudaGetErrorString(e));
  return r;
}

}  // namespace

extern "C" {

int dr_version(void) { return 100; }

const char* dr_last_error(void) { return g_err.c_str(); }

int dr_create(dr_ctx** out, int device, void* cuda_stream) {
  if (!out) return fail(DR_ERR_INVALID_ARG, "dr_create: out is NULL");
  *out = nullptr;
  int n = 0;
  DR_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(DR_ERR_INVALID_ARG, "dr_create: bad device index");
  DR_CUDA(cudaSetDevice(device));
  dr_ctx* c = new dr_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && n_sm > 0)
    c->n_sm = n_sm;
  cudaGetLastError();
  int r = dalloc(&c->counters, 4);
  if (r == DR_OK) r = dalloc(&c->err, 1);
  if (r == DR_OK) r = dalloc(&c->p_sum, 1);
  if (r == DR_OK) r = dalloc(&c->frame_dev, 1);
  if (r != DR_OK) {
    dr_destroy(c);
    return r;
  }
  cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), c->stream);
  cudaMemsetAsync(c->err, 0, sizeof(uint32_t), c->stream);
  *out = c;
  return check_launch("dr_create");
}

int dr_destroy(dr_ctx* c) {
  if (!c) return DR_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  dfree(&c->nodes4); dfree(&c->tris4);
  dfree(&c->nodes8); dfree(&c->tris8);
  free_two_level(c);
  dfree(&c->nodes); dfree(&c->tris); dfree(&c->surf); dfree(&c->lights); dfree(&c->nrm); dfree(&c->mats);
  dfree(&c->mw); dfree(&c->mmu); dfree(&c->msig);
  dfree(&c->x); dfree(&c->score); dfree(&c->logp); dfree(&c->killed);
  dfree(&c->xp); dfree(&c->sp); dfree(&c->cur);
  dfree(&c->plen); dfree(&c->order_a); dfree(&c->order_b);
  if (c->wf_mem) cudaFree(c->wf_mem); dfree(&c->rec); dfree(&c->rec_alt);
  if (c->sort_scratch) cudaFree(c->sort_scratch);
  dfree(&c->accum); dfree(&c->counters); dfree(&c->p_partial); dfree(&c->p_sum); dfree(&c->err);
  dfree(&c->frame_dev);
  free_batch(c);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (auto& m : c->marks) {
    cudaEventDestroy(m.begin);
    cudaEventDestroy(m.end);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->open_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return DR_OK;
}

int dr_scene_upload(dr_ctx* c, const float* verts, int32_t nv, const int32_t* tris, const float* normals, int32_t nt,
                    const int32_t* tri_mat, const float* mats, int32_t nm, const float* camera, int32_t width,
                    int32_t height) {
  if (!c || !verts || !tris || !tri_mat || !mats || !camera)
    return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: NULL argument");
  if (nv < 1 || nt < 1 || nm < 1 || width < 1 || height < 1 || (long long)width * height >= (1ll << 31))
    return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: bad size");
  // one parallel pass over the triangles (index and material checks, the
  // emitting ones with their power) and one over the vertices (finite,
  // extent); the light list keeps the triangle order
  struct TriPart {
    bool bad_index = false, bad_mat = false;
    std::vector<int> lt;
    std::vector<double> pw;
  };
  struct VertPart {
    bool bad = false;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  };
  std::vector<TriPart> tp(16);
  std::vector<VertPart> vp(16);
  auto V = [&](int i) { return f3(verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]); };
  const int ntp = parallel_parts(nt, [&](long long b, long long e, int p) {
    TriPart& q = tp[p];
    for (long long i = b; i < e; ++i) {
      const int i0 = tris[3 * i], i1 = tris[3 * i + 1], i2 = tris[3 * i + 2];
      if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
        q.bad_index = true;
        continue;
      }
      if (tri_mat[i] < 0 || tri_mat[i] >= nm) {
        q.bad_mat = true;
        continue;
      }
      const float* m = mats + 12 * tri_mat[i];
      if (!(m[6] > 0.f || m[7] > 0.f || m[8] > 0.f)) continue;
      const float3 a = V(i0), bb = V(i1), cc = V(i2);
      const float3 N = cross(bb - a, cc - a);
      const double area = 0.5 * std::sqrt((double)dot(N, N));
      const double pwr = area * (0.2126 * m[6] + 0.7152 * m[7] + 0.0722 * m[8]);
      if (!(pwr > 0.0)) continue;
      q.lt.push_back((int)i);
      q.pw.push_back(pwr);
    }
  });
  const int nvp = parallel_parts(nv, [&](long long b, long long e, int p) {
    VertPart& q = vp[p];
    for (long long i = b; i < e; ++i)
      for (int a = 0; a < 3; ++a) {
        const float v = verts[3 * i + a];
        if (!std::isfinite(v)) q.bad = true;
        q.lo[a] = std::min(q.lo[a], (double)v);
        q.hi[a] = std::max(q.hi[a], (double)v);
      }
  });
  for (int p = 0; p < ntp; ++p)
    if (tp[p].bad_index) return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: vertex index out of range");
  for (int p = 0; p < ntp; ++p)
    if (tp[p].bad_mat) return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: material out of range");
  for (int i = 0; i < nm; ++i) {
    const float t = mats[12 * i];
    if (!(t == 0.f || t == 1.f || t == 2.f || t == 3.f || t == 4.f))
      return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: bad material type");
    if ((t == 1.f || t == 4.f) && !(mats[12 * i + 4] > 0.f))
      return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: glossy / conductor roughness must be > 0");
    if (t == 4.f)
      for (int ch = 0; ch < 3; ++ch)
        if (!(mats[12 * i + 1 + ch] > 0.f) || !(mats[12 * i + 9 + ch] > 0.f) || !std::isfinite(mats[12 * i + 1 + ch]) ||
            !std::isfinite(mats[12 * i + 9 + ch]))
          return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: conductor eta and k must be finite and > 0");
    if (t == 2.f && !(mats[12 * i + 5] > 0.f)) return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: dielectric ior must be > 0");
  }
  for (int p = 0; p < nvp; ++p)
    if (vp[p].bad) return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: non-finite vertex");
  DR_CUDA(cudaSetDevice(c->device));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  // host-side scene constants: extent -> tmin, light table, camera basis
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int p = 0; p < nvp; ++p)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], vp[p].lo[a]);
      hi[a] = std::max(hi[a], vp[p].hi[a]);
    }
  const double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  std::vector<int> lt;
  std::vector<double> pw;
  double tot = 0.0;
  for (int p = 0; p < ntp; ++p) {
    lt.insert(lt.end(), tp[p].lt.begin(), tp[p].lt.end());
    pw.insert(pw.end(), tp[p].pw.begin(), tp[p].pw.end());
  }
  for (double x : pw) tot += x;
  std::vector<float> sel(nt, 0.f);
  std::vector<float4> lrec(4 * lt.size());
  double acc = 0.0;
  for (size_t k = 0; k < lt.size(); ++k) {
    const int i = lt[k];
    acc += pw[k];
    const float3 a = V(tris[3 * i]), b = V(tris[3 * i + 1]), cc = V(tris[3 * i + 2]);
    const float3 N = cross(b - a, cc - a);
    const float area = 0.5f * sqrtf(dot(N, N));
    sel[i] = (float)(pw[k] / tot);
    lrec[4 * k + 0] = make_float4(a.x, a.y, a.z, hbits_f(i));
    lrec[4 * k + 1] = make_float4(b.x, b.y, b.z, sel[i]);
    lrec[4 * k + 2] = make_float4(cc.x, cc.y, cc.z, area);
    const float* em = mats + 12 * tri_mat[i] + 6;
    lrec[4 * k + 3] = make_float4(k + 1 == lt.size() ? 1.0f : (float)(acc / tot), em[0], em[1], em[2]);
  }
  {
    const double eye[3] = {camera[0], camera[1], camera[2]}, look[3] = {camera[3], camera[4], camera[5]},
                 up[3] = {camera[6], camera[7], camera[8]};
    double fw[3] = {look[0] - eye[0], look[1] - eye[1], look[2] - eye[2]};
    double l = std::sqrt(fw[0] * fw[0] + fw[1] * fw[1] + fw[2] * fw[2]);
    if (!(l > 0.0) || !(camera[9] > 0.f && camera[9] < 180.f))
      return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: degenerate camera");
    for (double& v : fw) v /= l;
    double rt[3] = {fw[1] * up[2] - fw[2] * up[1], fw[2] * up[0] - fw[0] * up[2], fw[0] * up[1] - fw[1] * up[0]};
    l = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
    if (!(l > 0.0)) return fail(DR_ERR_INVALID_ARG, "dr_scene_upload: camera up parallel to view");
    for (double& v : rt) v /= l;
    const double u2[3] = {rt[1] * fw[2] - rt[2] * fw[1], rt[2] * fw[0] - rt[0] * fw[2], rt[0] * fw[1] - rt[1] * fw[0]};
    const double th = std::tan(0.5 * camera[9] * 3.14159265358979323846 / 180.0);
    c->cam.eye = f3(camera[0], camera[1], camera[2]);
    c->cam.fwd = f3((float)fw[0], (float)fw[1], (float)fw[2]);
    c->cam.right = f3((float)rt[0], (float)rt[1], (float)rt[2]);
    c->cam.up = f3((float)u2[0], (float)u2[1], (float)u2[2]);
    c->cam.ty = (float)th;
    c->cam.tx = (float)(th * width / height);
  }
  // Every check has passed: the old scene (target or batch) is replaced from
  // here on.  Until this upload succeeds the context has none, so no call
  // can reach a buffer that is freed or reallocated below.
  c->target = -1;
  c->inited = false;
  c->target_gen++;
  free_batch(c);
  free_two_level(c);
  // device arrays
  float* dverts = nullptr;
  int* dtris = nullptr;
  int* dmat = nullptr;
  float* dsel = nullptr;
  float* dvn = nullptr;
  void* scratch = nullptr;
  int r = DR_OK;
  const int n_nodes = std::max(1, nt - 1);
  r = dalloc(&dverts, 3 * (size_t)nv);
  if (r == DR_OK) r = dalloc(&dtris, 3 * (size_t)nt);
  if (r == DR_OK) r = dalloc(&dmat, (size_t)nt);
  if (r == DR_OK) r = dalloc(&dsel, (size_t)nt);
  if (r == DR_OK && normals) r = dalloc(&dvn, 3 * (size_t)nv);
  if (r == DR_OK) r = dalloc(&c->nodes, 4 * (size_t)n_nodes);
  if (r == DR_OK) r = dalloc(&c->tris, 3 * (size_t)nt);
  if (r == DR_OK) r = dalloc(&c->surf, 5 * (size_t)nt);
  if (r == DR_OK) r = dalloc(&c->mats, 12 * (size_t)nm);
  if (r == DR_OK) r = dalloc(&c->lights, std::max<size_t>(4, lrec.size()));
  if (r == DR_OK) r = normals ? dalloc(&c->nrm, 9 * (size_t)nt) : (dfree(&c->nrm), DR_OK);
  void* ploc_scratch = nullptr;
  if (r == DR_OK) {
    cudaError_t e = cudaMalloc(&scratch, bvh_scratch_bytes(nt));
    if (e == cudaSuccess && c->builder == DR_BVH_PLOC) e = cudaMalloc(&ploc_scratch, ploc_scratch_bytes(nt));
    if (e != cudaSuccess) { cudaGetLastError(); r = fail(DR_ERR_OOM, "dr_scene_upload: BVH scratch"); }
  }
  if (r == DR_OK) {
    cudaStream_t s = c->stream;
    cudaMemcpyAsync(dverts, verts, 12 * (size_t)nv, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dtris, tris, 12 * (size_t)nt, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dmat, tri_mat, 4 * (size_t)nt, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dsel, sel.data(), 4 * (size_t)nt, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->mats, mats, 48 * (size_t)nm, cudaMemcpyHostToDevice, s);
    if (!lrec.empty()) cudaMemcpyAsync(c->lights, lrec.data(), 16 * lrec.size(), cudaMemcpyHostToDevice, s);
    if (normals) {
      cudaMemcpyAsync(dvn, normals, 12 * (size_t)nv, cudaMemcpyHostToDevice, s);
      launch_gather_normals(dvn, dtris, nt, c->nrm, s);
    }
    launch_surface_records(dverts, dtris, dmat, dsel, dvn, nt, c->surf, s);
    c->n_nodes = c->builder == DR_BVH_PLOC
                     ? build_ploc(dverts, dtris, nt, c->nodes, c->tris, scratch, ploc_scratch, c->ploc_radius,
                                  kTraversalStack + 1, s)
                     : build_lbvh(dverts, dtris, nt, c->nodes, c->tris, scratch, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) r = fail(DR_ERR_CUDA, std::string("dr_scene_upload: ") + cudaGetErrorString(e));
    else if (c->n_nodes < 0) r = fail(DR_ERR_CUDA, "dr_scene_upload: BVH construction failed");
  }
  dfree(&dverts); dfree(&dtris); dfree(&dmat); dfree(&dsel); dfree(&dvn);
  if (scratch) cudaFree(scratch);
  if (ploc_scratch) cudaFree(ploc_scratch);
  if (r != DR_OK) return r;
  c->target = 0;
  c->conductors = false;
  for (int i = 0; i < nm; ++i) c->conductors = c->conductors || mats[12 * i] == 4.f;
  c->W = width;
  c->H = height;
  c->nt = nt;
  c->n_lights = (int)lt.size();
  c->tmin = (float)(1e-5 * ext);
  c->inited = false;
  // the hierarchy must be a tree (checked on the device) that the
  // traversal stack can hold
  int depth = 1;
  r = build_bvh4(c, &depth);
  if (r == DR_OK) r = build_bvh8(c);
  if (r == DR_OK && depth - 1 > kTraversalStack)
    r = fail(DR_ERR_DEVICE_CHECK, "dr_scene_upload: BVH depth " + std::to_string(depth) +
                                      " exceeds the traversal stack (" + std::to_string(kTraversalStack + 1) + ")");
  if (r != DR_OK) c->target = -1;
  c->target_gen++;
  return r;
}

int dr_target_mixture(dr_ctx* c, int32_t d, int32_t K, const float* w, const float* mu, const float* sig, float cval,
                      int32_t width, int32_t height) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_target_mixture: NULL ctx");
  if (d < 2 || d > kMaxDim || (d & 1) || K < 0 || width < 1 || height < 1)
    return fail(DR_ERR_INVALID_ARG, "dr_target_mixture: bad size");
  if (K > 0 && (!w || !mu || !sig)) return fail(DR_ERR_INVALID_ARG, "dr_target_mixture: NULL arrays");
  for (int k = 0; k < K; ++k)
    if (!(sig[k] > 0.f)) return fail(DR_ERR_INVALID_ARG, "dr_target_mixture: sigma must be > 0");
  DR_CUDA(cudaSetDevice(c->device));
  // the old target is replaced from here on: until this call succeeds the
  // context has none (no call can reach a buffer freed below)
  c->target = -1;
  c->inited = false;
  c->target_gen++;
  free_batch(c);
  DR_TRY(dalloc(&c->mw, std::max(1, K)));
  DR_TRY(dalloc(&c->mmu, std::max(1, K * d)));
  DR_TRY(dalloc(&c->msig, std::max(1, K)));
  if (K > 0) {
    DR_CUDA(cudaMemcpyAsync(c->mw, w, 4 * (size_t)K, cudaMemcpyHostToDevice, c->stream));
    DR_CUDA(cudaMemcpyAsync(c->mmu, mu, 4 * (size_t)K * d, cudaMemcpyHostToDevice, c->stream));
    DR_CUDA(cudaMemcpyAsync(c->msig, sig, 4 * (size_t)K, cudaMemcpyHostToDevice, c->stream));
  }
  DR_CUDA(cudaStreamSynchronize(c->stream));
  c->target = 1;
  c->mK = K;
  c->md = d;
  c->mcval = cval;
  c->W = width;
  c->H = height;
  c->inited = false;
  c->target_gen++;
  return DR_OK;
}

static int validate_params(const dr_params* p) {
  if (!p) return fail(DR_ERR_INVALID_ARG, "params: NULL");
  if (p->max_path_len < 1 || p->max_path_len > DR_MAX_PATH_LEN) return fail(DR_ERR_INVALID_ARG, "params: max_path_len");
  if (p->drift_mode < 0 || p->drift_mode > 3) return fail(DR_ERR_INVALID_ARG, "params: drift_mode");
  if (!(p->stddev > 0.f) || !(p->dt > 0.f) || !(p->eps > 0.f) || !(p->m > 0.f))
    return fail(DR_ERR_INVALID_ARG, "params: stddev, dt, eps and m must be > 0");
  if (!std::isfinite(p->gamma_tilde)) return fail(DR_ERR_INVALID_ARG, "params: gamma_tilde");
  if (p->drift_mode == DR_DRIFT_FD && !(p->fd_h > 0.f && p->fd_h < 0.5f)) return fail(DR_ERR_INVALID_ARG, "params: fd_h");
  if (p->steps_per_splat < 1 || p->steps_per_splat > 4096) return fail(DR_ERR_INVALID_ARG, "params: steps_per_splat");
  return DR_OK;
}

static int alloc_chains_sized(dr_ctx* c, unsigned long long N, int d, int spp, bool mala) {
  const size_t nd = (size_t)N * d;
  if (nd > c->state_cap) {
    DR_TRY(dalloc(&c->x, nd));
    DR_TRY(dalloc(&c->score, nd));
    c->state_cap = nd;
  }
  if (N > c->chains_cap) {
    DR_TRY(dalloc(&c->logp, N));
    DR_TRY(dalloc(&c->killed, N));
    DR_TRY(dalloc(&c->plen, N));
    DR_TRY(dalloc(&c->order_a, N));
    DR_TRY(dalloc(&c->order_b, N));
    c->chains_cap = N;
  }
  const size_t nrec = (size_t)N * spp;
  if (nrec > c->rec_cap_records) {
    DR_TRY(dalloc(&c->rec, nrec));
    DR_TRY(dalloc(&c->rec_alt, nrec));
    if (c->sort_scratch) cudaFree(c->sort_scratch);
    c->sort_scratch = nullptr;
    cudaError_t e = cudaMalloc(&c->sort_scratch, sort_scratch_bytes(nrec));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->rec_cap_records = 0;
      return fail(DR_ERR_OOM, "sort scratch");
    }
    c->rec_cap_records = nrec;
  }
  if (mala && nd > c->mala_cap) {
    DR_TRY(dalloc(&c->xp, nd));
    DR_TRY(dalloc(&c->sp, nd));
    DR_TRY(dalloc(&c->cur, (size_t)N));
    c->mala_cap = nd;
  }
  const size_t npart = (N + step_block_size() - 1) / step_block_size();
  if (npart > c->p_partial_cap) {
    DR_TRY(dalloc(&c->p_partial, npart));
    c->p_partial_cap = npart;
  }
  const size_t na = (size_t)c->W * c->H * 3;
  if (na != c->accum_n) {
    DR_TRY(dalloc(&c->accum, na));
    c->accum_n = na;
  }
  return DR_OK;
}

// Sizes the chain buffers for an init.  The context has no chains until the
// caller's init succeeds (a failure here or later in the init leaves
// dr_step and the other chain calls refusing with STATE).  dalloc frees a
// buffer before it allocates the larger one, so a failed allocation forgets
// every capacity: the next init allocates afresh and no call can reach a
// freed or null buffer.
static int alloc_chains(dr_ctx* c, unsigned long long N, int d, int spp, bool mala = false) {
  c->inited = false;
  const int r = alloc_chains_sized(c, N, d, spp, mala);
  if (r != DR_OK) {
    c->state_cap = 0;
    c->mala_cap = 0;
    c->chains_cap = 0;
    c->rec_cap_records = 0;
    c->p_partial_cap = 0;
    c->accum_n = 0;
  }
  return r;
}

int dr_scenes_upload_batch(dr_ctx* c, const dr_scene_desc* sd, int32_t n) {
  if (!c || !sd) return fail(DR_ERR_INVALID_ARG, "dr_scenes_upload_batch: NULL argument");
  if (n < 1 || n > 255) return fail(DR_ERR_INVALID_ARG, "dr_scenes_upload_batch: n_scenes must be 1..255");
  for (int i = 0; i < n; ++i)
    if (sd[i].max_path_len < 1 || sd[i].max_path_len > DR_MAX_PATH_LEN || sd[i].n_chains < 1 ||
        sd[i].n_chains > (1ull << 31))
      return fail(DR_ERR_INVALID_ARG, "dr_scenes_upload_batch: scene " + std::to_string(i) +
                                          ": max_path_len 1..16 and n_chains 1..2^31");
  DR_CUDA(cudaSetDevice(c->device));
  free_batch(c);
  c->target = -1;
  c->inited = false;
  c->target_gen++;
  std::vector<DevScene> ds((size_t)n);
  unsigned long long pix = 0, chains = 0;
  long long tris = 0;
  for (int i = 0; i < n; ++i) {
    const dr_scene_desc& q = sd[i];
    dr_ctx* sub = nullptr;
    int r = dr_create(&sub, c->device, c->stream);
    if (r != DR_OK) {
      free_batch(c);
      return r;
    }
    sub->builder = c->builder;
    sub->ploc_radius = c->ploc_radius;
    sub->bvh_width = c->bvh_width == 8 ? 8 : 4;
    c->subs.push_back(sub);
    r = dr_scene_upload(sub, q.verts, q.nv, q.tris, q.normals, q.nt, q.tri_mat, q.mats, q.nm, q.camera, q.width,
                        q.height);
    if (r == DR_OK && !sub->nodes4)
      r = fail(DR_ERR_INVALID_ARG, "no 4-wide BVH (a batch scene needs at least 2 triangles)");
    if (r == DR_OK && pix + (unsigned long long)q.width * q.height >= (1ull << 31))
      r = fail(DR_ERR_INVALID_ARG, "the batch's images exceed 2^31 pixels");
    if (r != DR_OK) {
      const std::string msg = "dr_scenes_upload_batch: scene " + std::to_string(i) + ": " + g_err;
      free_batch(c);
      return fail(r, msg);
    }
    ds[(size_t)i] = dev_scene(sub);
    SceneChains sc{};
    sc.chain0 = chains;
    sc.n = q.n_chains;
    sc.L = q.max_path_len;
    sc.d = 2 + 4 * (q.max_path_len - 1);
    sc.pix0 = (uint32_t)pix;
    c->h_sc.push_back(sc);
    c->batch_w.push_back(q.width);
    c->batch_h.push_back(q.height);
    pix += (unsigned long long)q.width * q.height;
    chains += q.n_chains;
    tris += q.nt;
  }
  int r = dalloc(&c->d_scenes, (size_t)n);
  if (r == DR_OK && cudaMemcpyAsync(c->d_scenes, ds.data(), ds.size() * sizeof(DevScene), cudaMemcpyHostToDevice,
                                    c->stream) != cudaSuccess)
    r = fail(DR_ERR_CUDA, "dr_scenes_upload_batch: scene table copy");
  if (r == DR_OK && cudaStreamSynchronize(c->stream) != cudaSuccess)
    r = fail(DR_ERR_CUDA, "dr_scenes_upload_batch: synchronise");
  if (r != DR_OK) {
    free_batch(c);
    return r;
  }
  c->target = 2;
  c->conductors = false;
  c->batch_bvh8 = !c->subs.empty();
  for (dr_ctx* sub : c->subs) {
    c->conductors = c->conductors || sub->conductors;
    c->batch_bvh8 = c->batch_bvh8 && sub->nodes8 != nullptr;
  }
  c->W = (int)pix;  // the shared accumulator is one row of all scenes' pixels
  c->H = 1;
  c->nt = (int)std::min<long long>(tris, 1ll << 30);
  c->n_lights = 0;
  return DR_OK;
}

namespace {

// Initialize (Alg. 1) for a batch: as for one scene, with p_lambda and k0
// per scene (each scene's p summed over its own chains, in the fused
// kernel's block order from the scene's first chain).
int init_batch(dr_ctx* c, uint64_t n_chains, uint64_t seed, uint32_t frame, const dr_params* prm) {
  if (prm->drift_mode != DR_DRIFT_ADJOINT)
    return fail(DR_ERR_INVALID_ARG, "dr_chains_init: a batch runs with the adjoint drift (DR_DRIFT_ADJOINT)");
  const int ns = (int)c->h_sc.size();
  unsigned long long total = 0;
  int Lmax = 1;
  for (const SceneChains& q : c->h_sc) {
    total += q.n;
    Lmax = std::max(Lmax, q.L);
  }
  if (n_chains != total)
    return fail(DR_ERR_INVALID_ARG, "dr_chains_init: n_chains must equal the batch's total (" +
                                        std::to_string(total) + ")");
  const int d = 2 + 4 * (Lmax - 1);
  dr_params p = *prm;
  p.max_path_len = Lmax;
  DR_TRY(alloc_chains(c, total, d, p.steps_per_splat));
  c->N = total;
  c->d = d;
  c->prm = p;
  c->seed = seed;
  c->frame = frame;
  c->step = 0;
  c->rec_cap = p.steps_per_splat;
  c->rec_count = 0;
  c->k0 = 0.0;
  c->p_lambda = 0.0;
  cudaStream_t s = c->stream;
  std::vector<uint8_t> cs((size_t)total);
  for (int q = 0; q < ns; ++q)
    std::fill(cs.begin() + (long long)c->h_sc[q].chain0, cs.begin() + (long long)(c->h_sc[q].chain0 + c->h_sc[q].n),
              (uint8_t)q);
  dfree(&c->chain_scene);
  dfree(&c->batch_tours);
  dfree(&c->batch_psum);
  dfree(&c->d_sc);
  DR_TRY(dalloc(&c->chain_scene, (size_t)total));
  DR_TRY(dalloc(&c->batch_tours, (size_t)ns));
  DR_TRY(dalloc(&c->batch_psum, (size_t)ns));
  DR_TRY(dalloc(&c->d_sc, (size_t)ns));
  for (int q = 0; q < ns; ++q) {
    c->h_sc[q].tour_count = c->batch_tours + q;
    c->h_sc[q].k0 = prm->k0 > 0.0 ? prm->k0 : 0.0;
  }
  DR_CUDA(cudaMemcpyAsync(c->chain_scene, cs.data(), cs.size(), cudaMemcpyHostToDevice, s));
  DR_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc.data(), ns * sizeof(SceneChains), cudaMemcpyHostToDevice, s));
  DR_CUDA(cudaMemsetAsync(c->batch_tours, 0, ns * sizeof(unsigned long long), s));
  DR_CUDA(cudaMemsetAsync(c->score, 0, (size_t)total * d * 4, s));
  DR_CUDA(cudaMemsetAsync(c->killed, 0, (size_t)total, s));
  DR_CUDA(cudaMemsetAsync(c->plen, 0, (size_t)total, s));
  DR_CUDA(cudaMemsetAsync(c->accum, 0, c->accum_n * 8, s));
  DR_CUDA(cudaMemsetAsync(c->counters, 0, 4 * 8, s));
  DR_CUDA(cudaMemsetAsync(c->err, 0, 4, s));
  DR_CUDA(cudaStreamSynchronize(s));  // the host copies above are of stack memory
  DR_TRY(ensure_wavefront_buffers(c));
  c->inited = true;
  if (prm->k0 > 0.0) return one_step(c, true);
  const WfBuffers w = wf_carve(c->wf_mem, c->N, c->prm.max_path_len);
  float* p_tmp = reinterpret_cast<float*>(w.hit);  // free once the last bounce is shaded
  StepArgs a = step_args(c);
  a.init = 1;
  a.step = 0;
  a.rec = c->rec;
  a.plen = c->plen;
  const PhaseHook hook{phase_mark, c};
  c->launches += launch_wavefront_step(a, w, c->stats, c->n_sm, c->tune, hook, s, kWfInitEval, p_tmp);
  for (int q = 0; q < ns; ++q) {
    const SceneChains& sc = c->h_sc[q];
    launch_block_sums(p_tmp + sc.chain0, sc.n, c->p_partial, s);
    const int nb = (int)((sc.n + step_block_size() - 1) / step_block_size());
    launch_sum_doubles(c->p_partial, nb, c->batch_psum + q, s);
    c->launches += 2;
  }
  DR_TRY(check_launch("batch init evaluation"));
  std::vector<double> psum((size_t)ns);
  DR_CUDA(cudaMemcpyAsync(psum.data(), c->batch_psum, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
  DR_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < ns; ++q) {
    const double pl = psum[q] / (double)c->h_sc[q].n;
    if (!(pl > 0.0) || !std::isfinite(pl)) {
      c->inited = false;
      return fail(DR_ERR_STATE, "dr_chains_init: estimated p_lambda of scene " + std::to_string(q) +
                                    " is not positive");
    }
    c->h_sc[q].k0 = pl / ((double)prm->m * (double)prm->dt);
  }
  DR_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc.data(), ns * sizeof(SceneChains), cudaMemcpyHostToDevice, s));
  c->launches += launch_wavefront_step(a, w, c->stats, c->n_sm, c->tune, hook, s, kWfInitClock, p_tmp);
  DR_TRY(check_launch("batch init clock"));
  DR_CUDA(cudaStreamSynchronize(s));
  c->rec_count = 1;
  return check_device_error(c);
}

}  // namespace

int dr_resolve_scene(dr_ctx* c, int32_t scene, float* out_rgb) {
  if (!c || !out_rgb) return fail(DR_ERR_INVALID_ARG, "dr_resolve_scene: NULL argument");
  if (c->target != 2) return fail(DR_ERR_STATE, "dr_resolve_scene: no batch uploaded");
  if (scene < 0 || scene >= (int)c->h_sc.size()) return fail(DR_ERR_INVALID_ARG, "dr_resolve_scene: scene index");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_resolve_scene: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(flush(c));
  const SceneChains& q = c->h_sc[scene];
  launch_resolve(c->accum + 3 * (size_t)q.pix0, 3 * (size_t)c->batch_w[scene] * c->batch_h[scene],
                 c->batch_tours + scene, q.k0, out_rgb, c->stream);
  c->launches += 1;
  DR_TRY(check_launch("resolve"));
  if (!capturing(c->stream)) {
    unsigned long long tc = 0;
    DR_CUDA(cudaMemcpyAsync(&tc, c->batch_tours + scene, 8, cudaMemcpyDeviceToHost, c->stream));
    DR_CUDA(cudaStreamSynchronize(c->stream));
    if (tc == 0) return fail(DR_ERR_STATE, "dr_resolve_scene: tourCount is 0 (no completed tour yet)");
  }
  return DR_OK;
}

int dr_get_scene_counters(dr_ctx* c, int32_t scene, uint64_t* tour_count, double* k0) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_get_scene_counters: NULL ctx");
  if (c->target != 2) return fail(DR_ERR_STATE, "dr_get_scene_counters: no batch uploaded");
  if (scene < 0 || scene >= (int)c->h_sc.size()) return fail(DR_ERR_INVALID_ARG, "dr_get_scene_counters: scene");
  DR_CUDA(cudaSetDevice(c->device));
  unsigned long long tc = 0;
  if (c->batch_tours) {
    DR_CUDA(cudaMemcpyAsync(&tc, c->batch_tours + scene, 8, cudaMemcpyDeviceToHost, c->stream));
    DR_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (tour_count) *tour_count = tc;
  if (k0) *k0 = c->h_sc[scene].k0;
  return check_device_error(c);
}

int dr_chains_init(dr_ctx* c, uint64_t n_chains, uint64_t seed, uint32_t frame, const dr_params* prm) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_chains_init: NULL ctx");
  DR_TRY(validate_params(prm));
  if (c->target < 0) return fail(DR_ERR_STATE, "dr_chains_init: no scene or target uploaded");
  if (c->target == 2) {
    DR_CUDA(cudaSetDevice(c->device));
    return init_batch(c, n_chains, seed, frame, prm);
  }
  if (n_chains < 1 || n_chains > (1ull << 31)) return fail(DR_ERR_INVALID_ARG, "dr_chains_init: n_chains");
  if (frame >= (1u << 28)) return fail(DR_ERR_INVALID_ARG, "dr_chains_init: frame must be < 2^28");
  const int d = c->target == 0 ? 2 + 4 * (prm->max_path_len - 1) : c->md;
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(alloc_chains(c, n_chains, d, prm->steps_per_splat, prm->drift_mode == DR_DRIFT_MALA));
  c->N = n_chains;
  c->d = d;
  c->prm = *prm;
  c->seed = seed;
  c->frame = frame;
  c->step = 0;
  c->rec_cap = prm->steps_per_splat;
  c->rec_count = 0;
  cudaStream_t s = c->stream;
  DR_CUDA(cudaMemsetAsync(c->score, 0, (size_t)n_chains * d * 4, s));
  DR_CUDA(cudaMemsetAsync(c->killed, 0, (size_t)n_chains, s));
  DR_CUDA(cudaMemsetAsync(c->plen, 0, (size_t)n_chains, s));
  DR_CUDA(cudaMemsetAsync(c->accum, 0, c->accum_n * 8, s));
  DR_CUDA(cudaMemsetAsync(c->counters, 0, 4 * 8, s));
  DR_CUDA(cudaMemsetAsync(c->err, 0, 4, s));
  c->p_lambda = 0.0;
  c->p_init_n = 0;
  if (prm->k0 <= 0.0 && use_wavefront(c)) {
    // one evaluation serves the p_lambda estimate and Init: evaluate (with
    // the adjoint for every chain), reduce p, then run the clock
    DR_TRY(ensure_wavefront_buffers(c));
    const WfBuffers w = wf_carve(c->wf_mem, c->N, c->prm.max_path_len);
    float* p_tmp = reinterpret_cast<float*>(w.hit);  // free once the last bounce is shaded
    StepArgs a = step_args(c);
    a.init = 1;
    a.step = 0;
    a.rec = c->rec;
    a.plen = c->plen;
    const PhaseHook hook{phase_mark, c};
    c->launches += launch_wavefront_step(a, w, c->stats, c->n_sm, c->tune, hook, s, kWfInitEval, p_tmp);
    launch_block_sums(p_tmp, n_chains, c->p_partial, s);
    const int nb = (int)((n_chains + step_block_size() - 1) / step_block_size());
    launch_sum_doubles(c->p_partial, nb, c->p_sum, s);
    c->launches += 2;
    DR_TRY(check_launch("init evaluation"));
    double sum = 0.0;
    DR_CUDA(cudaMemcpyAsync(&sum, c->p_sum, 8, cudaMemcpyDeviceToHost, s));
    DR_CUDA(cudaStreamSynchronize(s));
    c->p_lambda = sum / (double)n_chains;
    if (!(c->p_lambda > 0.0) || !std::isfinite(c->p_lambda))
      return fail(DR_ERR_STATE, "dr_chains_init: estimated p_lambda is not positive");
    c->p_init_sum = sum;
    c->p_init_n = n_chains;
    c->k0 = c->p_lambda / ((double)prm->m * (double)prm->dt);
    a.k0 = c->k0;
    c->launches += launch_wavefront_step(a, w, c->stats, c->n_sm, c->tune, hook, s, kWfInitClock, p_tmp);
    DR_TRY(check_launch("init clock"));
    c->inited = true;
    c->rec_count = 1;
    return check_device_error(c);
  }
  if (prm->k0 > 0.0) {
    c->k0 = prm->k0;
  } else {
    StepArgs a = step_args(c);
    a.init = 1;
    a.estimate_only = 1;
    a.step = 0;
    a.rec = nullptr;
    a.tour_count = nullptr;
    a.p_partial = c->p_partial;
    launch_step(a, false, s);
    DR_TRY(check_launch("init estimate"));
    const int nb = (int)((n_chains + step_block_size() - 1) / step_block_size());
    launch_sum_doubles(c->p_partial, nb, c->p_sum, s);
    double sum = 0.0;
    DR_CUDA(cudaMemcpyAsync(&sum, c->p_sum, 8, cudaMemcpyDeviceToHost, s));
    DR_CUDA(cudaStreamSynchronize(s));
    c->p_lambda = sum / (double)n_chains;
    if (!(c->p_lambda > 0.0) || !std::isfinite(c->p_lambda))
      return fail(DR_ERR_STATE, "dr_chains_init: estimated p_lambda is not positive");
    c->p_init_sum = sum;
    c->p_init_n = n_chains;
    c->k0 = c->p_lambda / ((double)prm->m * (double)prm->dt);
    DR_CUDA(cudaMemsetAsync(c->counters, 0, 4 * 8, s));
  }
  c->inited = true;
  DR_TRY(one_step(c, true));
  return DR_OK;
}

int dr_step(dr_ctx* c, uint32_t n_steps) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_step: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_step: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  for (uint32_t i = 0; i < n_steps; ++i) {
    c->step++;
    DR_TRY(one_step(c, false));
  }
  return DR_OK;
}

int dr_splat(dr_ctx* c) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_splat: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_splat: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  return flush(c);
}

int dr_resolve(dr_ctx* c, float* out_rgb) {
  if (!c || !out_rgb) return fail(DR_ERR_INVALID_ARG, "dr_resolve: NULL argument");
  if (c->target == 2) return fail(DR_ERR_STATE, "dr_resolve: a batch resolves per scene (dr_resolve_scene)");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_resolve: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(flush(c));
  launch_resolve(c->accum, c->accum_n, c->counters, c->k0, out_rgb, c->stream);
  c->launches += 1;
  DR_TRY(check_launch("resolve"));
  if (!capturing(c->stream)) {
    unsigned long long tc = 0;
    DR_CUDA(cudaMemcpyAsync(&tc, c->counters, 8, cudaMemcpyDeviceToHost, c->stream));
    DR_CUDA(cudaStreamSynchronize(c->stream));
    if (tc == 0) return fail(DR_ERR_STATE, "dr_resolve: tourCount is 0 (no completed tour yet)");
  }
  return DR_OK;
}

int dr_resolve_accum(const double* accum, int64_t n, uint64_t tour_count, double k0, float* out, void* cuda_stream) {
  if ((!accum || !out) && n > 0) return fail(DR_ERR_INVALID_ARG, "dr_resolve_accum: NULL argument");
  if (n < 0 || !std::isfinite(k0)) return fail(DR_ERR_INVALID_ARG, "dr_resolve_accum: n < 0 or k0 not finite");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  launch_resolve_count(accum, (size_t)n, (unsigned long long)tour_count, k0, out, s);
  DR_TRY(check_launch("resolve_accum"));
  if (tour_count == 0) return fail(DR_ERR_STATE, "dr_resolve_accum: tour_count is 0 (zero image written)");
  return DR_OK;
}

int dr_get_p_sum(dr_ctx* c, double* p_sum, uint64_t* n) {
  if (!c || !p_sum || !n) return fail(DR_ERR_INVALID_ARG, "dr_get_p_sum: NULL argument");
  if (!c->inited || c->p_init_n == 0)
    return fail(DR_ERR_STATE, "dr_get_p_sum: no p_lambda estimate (k0 was given or the chains were loaded)");
  *p_sum = c->p_init_sum;
  *n = c->p_init_n;
  return DR_OK;
}

int dr_k0_from_p_sum(double p_sum, uint64_t n, const dr_params* prm, double* k0) {
  if (!prm || !k0) return fail(DR_ERR_INVALID_ARG, "dr_k0_from_p_sum: NULL argument");
  const double mdt = (double)prm->m * (double)prm->dt;
  if (n == 0 || !(p_sum > 0.0) || !std::isfinite(p_sum) || !(mdt > 0.0) || !std::isfinite(mdt))
    return fail(DR_ERR_INVALID_ARG, "dr_k0_from_p_sum: n = 0, p_sum not positive, or m dt not positive");
  *k0 = p_sum / (double)n / mdt;
  return DR_OK;
}

int dr_readback_state(dr_ctx* c, float* x, float* score, uint8_t* killed, float* logp, int32_t* pix, float* val) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_readback_state: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_readback_state: chains not initialised");
  if ((pix || val) && c->rec_count == 0)
    return fail(DR_ERR_STATE, "dr_readback_state: last records were already splatted");
  DR_CUDA(cudaSetDevice(c->device));
  const size_t N = c->N, d = c->d;
  std::vector<float> tmp;
  auto soa = [&](const float* src, float* dst) -> int {
    tmp.resize(N * d);
    DR_CUDA(cudaMemcpyAsync(tmp.data(), src, N * d * 4, cudaMemcpyDeviceToHost, c->stream));
    DR_CUDA(cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < d; ++i)
      for (size_t j = 0; j < N; ++j) dst[j * d + i] = tmp[i * N + j];
    return DR_OK;
  };
  if (x) DR_TRY(soa(c->x, x));
  if (score) DR_TRY(soa(c->score, score));
  if (killed) DR_CUDA(cudaMemcpyAsync(killed, c->killed, N, cudaMemcpyDeviceToHost, c->stream));
  if (logp) DR_CUDA(cudaMemcpyAsync(logp, c->logp, N * 4, cudaMemcpyDeviceToHost, c->stream));
  if (pix || val) {
    std::vector<SplatRec> r(N);
    DR_CUDA(cudaMemcpyAsync(r.data(), c->rec + (size_t)(c->rec_count - 1) * N, N * sizeof(SplatRec),
                            cudaMemcpyDeviceToHost, c->stream));
    DR_CUDA(cudaStreamSynchronize(c->stream));
    for (size_t j = 0; j < N; ++j) {
      if (pix) pix[j] = (int32_t)r[j].pix;
      if (val) { val[3 * j] = r[j].r; val[3 * j + 1] = r[j].g; val[3 * j + 2] = r[j].b; }
    }
  }
  DR_CUDA(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

int dr_readback_accum(dr_ctx* c, double* accum) {
  if (!c || !accum) return fail(DR_ERR_INVALID_ARG, "dr_readback_accum: NULL argument");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_readback_accum: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(flush(c));
  DR_CUDA(cudaMemcpyAsync(accum, c->accum, c->accum_n * 8, cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

int dr_get_counters(dr_ctx* c, uint64_t* tour_count, double* k0, uint64_t* steps, uint64_t* rays, double* p_lambda) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_get_counters: NULL ctx");
  DR_CUDA(cudaSetDevice(c->device));
  unsigned long long h[4] = {0, 0, 0, 0};
  DR_CUDA(cudaMemcpyAsync(h, c->counters, 32, cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  if (tour_count) *tour_count = h[0];
  if (rays) *rays = h[1];
  if (k0) *k0 = c->k0;
  if (steps) *steps = c->step;
  if (p_lambda) *p_lambda = c->p_lambda;
  return check_device_error(c);
}

int dr_eval_logp(dr_ctx* c, int32_t L, const float* x, int64_t M, float* logp, float* grad, int32_t* pix, float* f) {
  if (!c || !x || !logp) return fail(DR_ERR_INVALID_ARG, "dr_eval_logp: NULL argument");
  if (c->target < 0 || c->target == 2) return fail(DR_ERR_STATE, "dr_eval_logp: no single scene or target");
  if (M < 0) return fail(DR_ERR_INVALID_ARG, "dr_eval_logp: M < 0");
  if (c->target == 0 && (L < 1 || L > DR_MAX_PATH_LEN)) return fail(DR_ERR_INVALID_ARG, "dr_eval_logp: L");
  DR_CUDA(cudaSetDevice(c->device));
  EvalArgs a{};
  a.S = dev_scene(c);
  a.M = dev_mixture(c);
  a.target = c->target;
  a.x = x;
  a.logp = logp;
  a.grad = grad;
  a.pix = pix;
  a.f = f;
  a.Mpts = M;
  a.d = c->target == 0 ? 2 + 4 * (L - 1) : c->md;
  a.L = L;
  a.eps = c->inited ? c->prm.eps : 1e-8f;
  a.err = c->err;
  launch_eval(a, c->stream);
  return check_launch("eval_logp");
}

int dr_lstar_over_p(dr_ctx* c, const dr_params* prm, const float* y, int64_t M, float radius, int32_t n,
                    double* out) {
  if (!c || !prm || ((!y || !out) && M > 0)) return fail(DR_ERR_INVALID_ARG, "dr_lstar_over_p: NULL argument");
  if (M < 0 || !(radius > 0.0f) || n < 2 || n > 4097)
    return fail(DR_ERR_INVALID_ARG, "dr_lstar_over_p: M < 0, radius <= 0 or n outside 2..4097");
  if (!(prm->stddev > 0.f) || !(prm->dt > 0.f) || !(prm->eps > 0.f) || !std::isfinite(prm->gamma_tilde))
    return fail(DR_ERR_INVALID_ARG, "dr_lstar_over_p: stddev, dt, eps must be > 0 and gamma_tilde finite");
  if (c->target != 1 || c->md != 2) return fail(DR_ERR_STATE, "dr_lstar_over_p: needs a mixture target on T^2");
  if (M == 0) return DR_OK;
  DR_CUDA(cudaSetDevice(c->device));
  LstarArgs a{};
  a.M = dev_mixture(c);
  a.y = y;
  a.n_pts = M;
  a.stddev = prm->stddev;
  a.h = 1.0 / (double)prm->dt;
  a.gamma_tilde = prm->gamma_tilde;
  a.eps = prm->eps;
  a.radius = radius;
  a.n = n;
  a.out = out;
  launch_lstar(a, c->stream);
  c->launches += 1;
  return check_launch("lstar_over_p");
}

int dr_trace_closest(dr_ctx* c, const float* rays, int64_t n, int32_t exclude, int32_t* tri, float* t) {
  if (!c || !rays || !tri || !t) return fail(DR_ERR_INVALID_ARG, "dr_trace_closest: NULL argument");
  if (n < 0) return fail(DR_ERR_INVALID_ARG, "dr_trace_closest: n < 0");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_trace_closest: no scene");
  DR_CUDA(cudaSetDevice(c->device));
  launch_trace(dev_scene(c), rays, n, exclude, tri, t, c->err, c->stream);
  return check_launch("trace_closest");
}

int dr_trace_closest_counted(dr_ctx* c, const float* rays, int64_t n, int32_t exclude, int32_t* tri, float* t,
                             uint32_t* node_steps, uint32_t* tri_tests) {
  if (!c || !rays || !tri || !t || !node_steps || !tri_tests)
    return fail(DR_ERR_INVALID_ARG, "dr_trace_closest_counted: NULL argument");
  if (n < 0) return fail(DR_ERR_INVALID_ARG, "dr_trace_closest_counted: n < 0");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_trace_closest_counted: no scene");
  DR_CUDA(cudaSetDevice(c->device));
  launch_trace_stats(dev_scene(c), rays, n, exclude, tri, t, node_steps, tri_tests, c->err, c->stream);
  return check_launch("trace_closest_counted");
}

int dr_bvh4_download(dr_ctx* c, float* nodes, float* tris) {
  if (!c || !nodes || !tris) return fail(DR_ERR_INVALID_ARG, "dr_bvh4_download: NULL argument");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_bvh4_download: no scene");
  if (!c->nodes4) return fail(DR_ERR_STATE, "dr_bvh4_download: the scene has no 4-wide BVH");
  DR_CUDA(cudaSetDevice(c->device));
  DR_CUDA(cudaMemcpyAsync(nodes, c->nodes4, (size_t)c->n_nodes4 * kNode4F4 * sizeof(float4), cudaMemcpyDeviceToHost,
                          c->stream));
  DR_CUDA(cudaMemcpyAsync(tris, c->tris4, (size_t)c->nt * kTriF4 * sizeof(float4), cudaMemcpyDeviceToHost,
                          c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  return DR_OK;
}

int dr_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream) {
  if (!ctr || !key || !out || n < 0) return fail(DR_ERR_INVALID_ARG, "dr_philox: bad argument");
  launch_philox(ctr, key, out, n, static_cast<cudaStream_t>(stream));
  return check_launch("philox");
}

int dr_splat_records(dr_ctx* c, const void* recs, int64_t M) {
  if (!c || (!recs && M > 0) || M < 0) return fail(DR_ERR_INVALID_ARG, "dr_splat_records: bad argument");
  if (c->accum_n == 0) return fail(DR_ERR_STATE, "dr_splat_records: no image (init chains first)");
  if (M == 0) return DR_OK;
  DR_CUDA(cudaSetDevice(c->device));
  SplatRec* a = nullptr;
  SplatRec* b = nullptr;
  uint32_t* bad = nullptr;  // this call's own check word: a bad record fails this call only
  void* scratch = nullptr;
  int r = dalloc(&a, (size_t)M);
  if (r == DR_OK) r = dalloc(&b, (size_t)M);
  if (r == DR_OK) r = dalloc(&bad, 1);
  if (r == DR_OK && cudaMalloc(&scratch, sort_scratch_bytes((size_t)M)) != cudaSuccess) {
    cudaGetLastError();
    scratch = nullptr;
    r = fail(DR_ERR_OOM, "dr_splat_records: scratch");
  }
  if (r == DR_OK) {
    cudaError_t e = cudaMemcpyAsync(a, recs, (size_t)M * sizeof(SplatRec), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) {
      SplatRec* sorted = sort_splat_records(a, b, (size_t)M, key_bits((long long)c->W * c->H), scratch, c->stream);
      launch_segment_reduce(sorted, (size_t)M, c->accum, (uint32_t)((size_t)c->W * c->H), bad, c->stream);
      e = cudaStreamSynchronize(c->stream);
      if (e == cudaSuccess) e = cudaGetLastError();
    } else {
      cudaGetLastError();
    }
    uint32_t flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, bad, sizeof(flags), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) r = fail(DR_ERR_CUDA, std::string("dr_splat_records: ") + cudaGetErrorString(e));
    else if (flags) r = fail(DR_ERR_DEVICE_CHECK, "dr_splat_records: a record's pixel index is >= W * H");
  }
  dfree(&a);
  dfree(&b);
  dfree(&bad);
  if (scratch) cudaFree(scratch);
  return r;
}

int dr_clear_image(dr_ctx* c) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_clear_image: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_clear_image: chains not initialised");
  DR_CUDA(cudaSetDevice(c->device));
  c->rec_count = 0;
  DR_CUDA(cudaMemsetAsync(c->accum, 0, c->accum_n * 8, c->stream));
  DR_CUDA(cudaMemsetAsync(c->counters, 0, 8, c->stream));
  return DR_OK;
}

namespace {
struct SaveHeader {
  uint64_t magic, version, N, seed, step;
  int32_t d, W, H, frame;
  dr_params prm;
  double k0, p_lambda;
  uint64_t counters[4];
};
constexpr uint64_t kMagic = 0x3152545345524644ull;  // "DFRESTR1"
}  // namespace

int dr_state_save(dr_ctx* c, void* host_buf, size_t* bytes) {
  if (!c || !bytes) return fail(DR_ERR_INVALID_ARG, "dr_state_save: NULL argument");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_state_save: chains not initialised");
  if (c->target == 2) return fail(DR_ERR_STATE, "dr_state_save: not available for a batch");
  if (c->prm.drift_mode == DR_DRIFT_MALA)
    return fail(DR_ERR_STATE, "dr_state_save: MALA chains (their current-state records) are not checkpointed");
  const size_t nd = (size_t)c->N * c->d;
  const size_t need = sizeof(SaveHeader) + nd * 8 + c->N * 5 + c->accum_n * 8;
  if (!host_buf) {
    *bytes = need;
    return DR_OK;
  }
  if (*bytes < need) return fail(DR_ERR_INVALID_ARG, "dr_state_save: buffer too small");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(flush(c));
  SaveHeader h{};
  h.magic = kMagic;
  h.version = 1;
  h.N = c->N;
  h.seed = c->seed;
  h.step = c->step;
  h.d = c->d;
  h.W = c->W;
  h.H = c->H;
  h.frame = (int32_t)c->frame;
  h.prm = c->prm;
  h.k0 = c->k0;
  h.p_lambda = c->p_lambda;
  DR_CUDA(cudaMemcpyAsync(h.counters, c->counters, 32, cudaMemcpyDeviceToHost, c->stream));
  char* p = static_cast<char*>(host_buf) + sizeof(SaveHeader);
  DR_CUDA(cudaMemcpyAsync(p, c->x, nd * 4, cudaMemcpyDeviceToHost, c->stream)); p += nd * 4;
  DR_CUDA(cudaMemcpyAsync(p, c->score, nd * 4, cudaMemcpyDeviceToHost, c->stream)); p += nd * 4;
  DR_CUDA(cudaMemcpyAsync(p, c->logp, c->N * 4, cudaMemcpyDeviceToHost, c->stream)); p += c->N * 4;
  DR_CUDA(cudaMemcpyAsync(p, c->killed, c->N, cudaMemcpyDeviceToHost, c->stream)); p += c->N;
  DR_CUDA(cudaMemcpyAsync(p, c->accum, c->accum_n * 8, cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  std::memcpy(host_buf, &h, sizeof(h));
  *bytes = need;
  return DR_OK;
}

int dr_state_load(dr_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return fail(DR_ERR_INVALID_ARG, "dr_state_load: NULL argument");
  if (bytes < sizeof(SaveHeader)) return fail(DR_ERR_INVALID_ARG, "dr_state_load: buffer too small");
  if (c->target == 2) return fail(DR_ERR_STATE, "dr_state_load: not available for a batch");
  SaveHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kMagic || h.version != 1) return fail(DR_ERR_INVALID_ARG, "dr_state_load: not a checkpoint");
  if (c->target < 0) return fail(DR_ERR_STATE, "dr_state_load: upload the scene or target first");
  // every field that sizes a buffer or a launch is checked before use, with
  // the limits dr_chains_init applies
  DR_TRY(validate_params(&h.prm));
  if (h.N < 1 || h.N > (1ull << 31)) return fail(DR_ERR_INVALID_ARG, "dr_state_load: chain count out of range");
  if (!(h.k0 > 0.0) || !std::isfinite(h.k0)) return fail(DR_ERR_INVALID_ARG, "dr_state_load: k0");
  const int d = c->target == 0 ? 2 + 4 * (h.prm.max_path_len - 1) : c->md;
  if (d != h.d || h.W != c->W || h.H != c->H) return fail(DR_ERR_INVALID_ARG, "dr_state_load: shape mismatch");
  const size_t nd = (size_t)h.N * h.d;
  const size_t need = sizeof(SaveHeader) + nd * 8 + h.N * 5 + (size_t)h.W * h.H * 3 * 8;
  if (bytes < need) return fail(DR_ERR_INVALID_ARG, "dr_state_load: truncated checkpoint");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(alloc_chains(c, h.N, h.d, h.prm.steps_per_splat));
  c->N = h.N;
  c->d = h.d;
  c->prm = h.prm;
  c->seed = h.seed;
  c->frame = (uint32_t)h.frame;
  c->step = (uint32_t)h.step;
  c->k0 = h.k0;
  c->p_lambda = h.p_lambda;
  c->p_init_n = 0;
  c->rec_cap = h.prm.steps_per_splat;
  c->rec_count = 0;
  const char* p = static_cast<const char*>(host_buf) + sizeof(SaveHeader);
  DR_CUDA(cudaMemcpyAsync(c->x, p, nd * 4, cudaMemcpyHostToDevice, c->stream)); p += nd * 4;
  DR_CUDA(cudaMemcpyAsync(c->score, p, nd * 4, cudaMemcpyHostToDevice, c->stream)); p += nd * 4;
  DR_CUDA(cudaMemcpyAsync(c->logp, p, h.N * 4, cudaMemcpyHostToDevice, c->stream)); p += h.N * 4;
  DR_CUDA(cudaMemcpyAsync(c->killed, p, h.N, cudaMemcpyHostToDevice, c->stream)); p += h.N;
  DR_CUDA(cudaMemcpyAsync(c->accum, p, c->accum_n * 8, cudaMemcpyHostToDevice, c->stream));
  DR_CUDA(cudaMemcpyAsync(c->counters, h.counters, 32, cudaMemcpyHostToDevice, c->stream));
  DR_CUDA(cudaMemsetAsync(c->err, 0, 4, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  c->inited = true;
  return DR_OK;
}

namespace {

// Everything a captured frame's launches depend on: buffers, sizes,
// parameters and options.  A frame is recaptured when any of it changes.
// The step index, seed, frame number and k0 are not part of it: the graph
// reads them from device memory, so re-initialised chains replay it.
std::vector<unsigned long long> frame_key(const dr_ctx* c, uint32_t n_steps) {
  auto P = [](const void* p) { return (unsigned long long)(uintptr_t)p; };
  unsigned long long prm[6];
  std::memset(prm, 0, sizeof(prm));
  std::memcpy(prm, &c->prm, std::min(sizeof(prm), sizeof(c->prm)));
  std::vector<unsigned long long> k = {n_steps, c->N, (unsigned long long)c->d, (unsigned long long)c->target,
                                       P(c->x), P(c->score), P(c->killed), P(c->logp), P(c->plen), P(c->rec),
                                       P(c->rec_alt), P(c->sort_scratch), P(c->accum), P(c->wf_mem), P(c->nodes),
                                       P(c->nodes4), P(c->nodes8), P(c->tl_nodes), (unsigned long long)c->two_level,
                                       (unsigned long long)c->bvh_width, P(c->tris), P(c->surf), P(c->mats), P(c->lights), P(c->nrm), P(c->mw),
                                       c->rec_cap, (unsigned long long)c->wavefront,
                                       (unsigned long long)c->work_order, (unsigned long long)c->stats,
                                       (unsigned long long)c->nt, (unsigned long long)c->n_lights, P(c->stream),
                                       c->target_gen, P(c->d_scenes), P(c->d_sc), P(c->chain_scene),
                                       (unsigned long long)c->tune.blocks_per_sm,
                                       (unsigned long long)c->tune.refill, (unsigned long long)c->ray_order,
                                       (unsigned long long)(c->tail_bounce + 1)};
  for (unsigned long long v : prm) k.push_back(v);
  return k;
}

}  // namespace

int dr_frame(dr_ctx* c, uint32_t n_steps) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_frame: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_frame: chains not initialised");
  if (n_steps == 0) return DR_OK;
  if (c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
    return fail(DR_ERR_STATE, "dr_frame: needs a created (non-default) CUDA stream for graph capture");
  DR_CUDA(cudaSetDevice(c->device));
  DR_TRY(flush(c));  // a frame starts with an empty record buffer
  if (use_wavefront(c)) DR_TRY(ensure_wavefront_buffers(c));
  const std::vector<unsigned long long> key = frame_key(c, n_steps);
  if (!c->gexec || key != c->graph_key) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    const uint32_t saved_step = c->step;
    const unsigned long long saved_launches = c->launches;
    DR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    int r = DR_OK;
    for (uint32_t i = 0; i < n_steps && r == DR_OK; ++i) {
      c->step++;
      r = one_step(c, false);
    }
    if (r == DR_OK) r = flush(c);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->capturing = false;
    c->step = saved_step;
    c->rec_count = 0;
    c->graph_launches = c->launches - saved_launches;
    c->launches = saved_launches;
    if (r != DR_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return fail(DR_ERR_CUDA, std::string("dr_frame: capture failed: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->gexec = nullptr;
      return fail(DR_ERR_CUDA, std::string("dr_frame: instantiate: ") + cudaGetErrorString(ei));
    }
    c->graph_key = key;
  }
  // the graph reads the step index from device memory and advances it
  c->frame_host = FrameParams{c->step + 1, (uint32_t)c->seed, (uint32_t)(c->seed >> 32), c->frame, c->k0};
  DR_CUDA(cudaMemcpyAsync(c->frame_dev, &c->frame_host, sizeof(FrameParams), cudaMemcpyHostToDevice, c->stream));
  DR_CUDA(cudaGraphLaunch(c->gexec, c->stream));
  c->step += n_steps;
  c->launches += c->graph_launches;
  c->rec_count = 0;
  return DR_OK;
}

int dr_get_profile(dr_ctx* c, double* ms, uint64_t* counts, int32_t n) {
  if (!c || !ms || n < 1) return fail(DR_ERR_INVALID_ARG, "dr_get_profile: bad argument");
  DR_CUDA(cudaSetDevice(c->device));
  phase_collect(c);
  for (int i = 0; i < n; ++i) {
    ms[i] = i < kPhCount ? c->phase_ms[i] : 0.0;
    if (counts) counts[i] = i < kPhCount ? c->phase_n[i] : 0;
  }
  for (int i = 0; i < kPhCount; ++i) {
    c->phase_ms[i] = 0.0;
    c->phase_n[i] = 0;
  }
  std::memset(c->bounce_ms, 0, sizeof(c->bounce_ms));
  std::memset(c->bounce_rays, 0, sizeof(c->bounce_rays));
  return DR_OK;
}

int dr_get_bounce_profile(dr_ctx* c, double* ms, int32_t n_bounces) {
  if (!c || !ms || n_bounces < 1 || n_bounces > kMaxPathLen)
    return fail(DR_ERR_INVALID_ARG, "dr_get_bounce_profile: bad argument");
  DR_CUDA(cudaSetDevice(c->device));
  phase_collect(c);
  for (int row = 0; row < 3; ++row)
    for (int k = 1; k <= n_bounces; ++k) ms[row * n_bounces + k - 1] = c->bounce_ms[row][k];
  return DR_OK;
}

int dr_get_bounce_rays(dr_ctx* c, uint64_t* rays, int32_t n_bounces) {
  if (!c || !rays || n_bounces < 1 || n_bounces > kMaxPathLen)
    return fail(DR_ERR_INVALID_ARG, "dr_get_bounce_rays: bad argument");
  for (int row = 0; row < 2; ++row)
    for (int k = 1; k <= n_bounces; ++k) rays[row * n_bounces + k - 1] = c->bounce_rays[row][k];
  return DR_OK;
}

int dr_set_stats(dr_ctx* c, int enable) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_set_stats: NULL ctx");
  DR_CUDA(cudaSetDevice(c->device));
  c->stats = enable != 0;
  if (c->stats) {
    DR_CUDA(cudaMemsetAsync(c->counters + 1, 0, 24, c->stream));
  }
  return DR_OK;
}

int dr_get_traversal_stats(dr_ctx* c, uint64_t* node_visits, uint64_t* tri_tests, uint64_t* rays) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_get_traversal_stats: NULL ctx");
  DR_CUDA(cudaSetDevice(c->device));
  unsigned long long h[4];
  DR_CUDA(cudaMemcpyAsync(h, c->counters, 32, cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  if (rays) *rays = h[1];
  if (node_visits) *node_visits = h[2];
  if (tri_tests) *tri_tests = h[3];
  return DR_OK;
}

int dr_pt_render(dr_ctx* c, int32_t L, uint32_t spp, uint64_t seed, double* out_mean) {
  if (!c || !out_mean) return fail(DR_ERR_INVALID_ARG, "dr_pt_render: NULL argument");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_pt_render: no scene");
  if (L < 1 || L > DR_MAX_PATH_LEN || spp < 1) return fail(DR_ERR_INVALID_ARG, "dr_pt_render: bad L or spp");
  DR_CUDA(cudaSetDevice(c->device));
  const long long n_pix = (long long)c->W * c->H;
  // enough threads to fill the GPU, at most spp chunks
  long long want = (1ll << 20) / std::max(1ll, n_pix);
  const int n_chunks = (int)std::max(1ll, std::min<long long>(want, (long long)spp));
  double* part = nullptr;
  DR_TRY(dalloc(&part, (size_t)n_chunks * n_pix * 3));
  Rng rng{(uint32_t)seed, (uint32_t)(seed >> 32), 0u};
  launch_pt(dev_scene(c), L, spp, n_chunks, rng, part, out_mean, c->counters + 1, c->err, c->stream);
  c->launches += 2;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  dfree(&part);
  if (e != cudaSuccess) return fail(DR_ERR_CUDA, std::string("dr_pt_render: ") + cudaGetErrorString(e));
  return check_device_error(c);
}

int dr_set_option(dr_ctx* c, int32_t option, int32_t value) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_set_option: NULL ctx");
  switch (option) {
    case DR_OPT_PROFILE:
      if (value != 0 && value != 1) return fail(DR_ERR_INVALID_ARG, "dr_set_option: profile is 0 or 1");
      c->profile = value != 0;
      return DR_OK;
    case DR_OPT_WAVEFRONT:
      if (value < -1 || value > 1) return fail(DR_ERR_INVALID_ARG, "dr_set_option: wavefront is -1, 0 or 1");
      c->wavefront = value;
      return DR_OK;
    case DR_OPT_WORK_ORDER:
      if (value != 0 && value != 1) return fail(DR_ERR_INVALID_ARG, "dr_set_option: work order is 0 or 1");
      c->work_order = value;
      return DR_OK;
    case DR_OPT_TRAVERSE_BLOCKS:
      if (value < 0 || value > 64) return fail(DR_ERR_INVALID_ARG, "dr_set_option: traverse blocks is 0..64");
      c->tune.blocks_per_sm = value;
      return DR_OK;
    case DR_OPT_REFILL:
      if (value < 1 || value > 32) return fail(DR_ERR_INVALID_ARG, "dr_set_option: refill is 1..32");
      c->tune.refill = value;
      return DR_OK;
    case DR_OPT_TAIL_BOUNCE:
      if (value < -1 || value > DR_MAX_PATH_LEN) return fail(DR_ERR_INVALID_ARG, "dr_set_option: tail bounce is -1..16");
      c->tail_bounce = value;
      return DR_OK;
    case DR_OPT_RAY_ORDER:
      if (value < -1 || value > 1) return fail(DR_ERR_INVALID_ARG, "dr_set_option: ray order is -1, 0 or 1");
      c->ray_order = value;
      return DR_OK;
    case DR_OPT_TWO_LEVEL:
      if (value != 0 && value != 1) return fail(DR_ERR_INVALID_ARG, "dr_set_option: two-level is 0 or 1");
      c->two_level = value;
      return DR_OK;
    case DR_OPT_BVH_WIDTH:
      if (value != 0 && value != 2 && value != 4 && value != 8)
        return fail(DR_ERR_INVALID_ARG, "dr_set_option: BVH width is 0, 2, 4 or 8");
      c->bvh_width = value;
      return DR_OK;
    default:
      return fail(DR_ERR_INVALID_ARG, "dr_set_option: unknown option");
  }
}

int dr_set_bvh_builder(dr_ctx* c, int32_t builder, int32_t radius) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_set_bvh_builder: NULL ctx");
  if (builder != DR_BVH_LBVH && builder != DR_BVH_PLOC) return fail(DR_ERR_INVALID_ARG, "dr_set_bvh_builder: builder");
  if (builder == DR_BVH_PLOC && (radius < 1 || radius > 256))
    return fail(DR_ERR_INVALID_ARG, "dr_set_bvh_builder: radius must be 1..256");
  c->builder = builder;
  c->ploc_radius = radius;
  return DR_OK;
}

int dr_get_chain_shape(dr_ctx* c, uint64_t* n_chains, int32_t* dim, int32_t* max_path_len) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_get_chain_shape: NULL ctx");
  if (!c->inited) return fail(DR_ERR_STATE, "dr_get_chain_shape: no chains");
  if (n_chains) *n_chains = c->N;
  if (dim) *dim = c->d;
  if (max_path_len) *max_path_len = c->prm.max_path_len;
  return DR_OK;
}

int dr_get_launch_count(dr_ctx* c, uint64_t* launches) {
  if (!c || !launches) return fail(DR_ERR_INVALID_ARG, "dr_get_launch_count: NULL argument");
  *launches = c->launches;
  return DR_OK;
}

int dr_bvh4_info(dr_ctx* c, int32_t* n_nodes, int32_t* max_depth, int32_t* stack_need) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_bvh4_info: NULL ctx");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_bvh4_info: no scene");
  if (!c->nodes4) return fail(DR_ERR_STATE, "dr_bvh4_info: the scene has no 4-wide BVH");
  if (n_nodes) *n_nodes = c->n_nodes4;
  if (max_depth) *max_depth = c->bvh4_depth;
  if (stack_need) *stack_need = c->bvh4_stack;
  return DR_OK;
}

int dr_scene_upload_instanced(dr_ctx* c, const dr_mesh_desc* meshes, int32_t n_meshes,
                              const dr_instance_desc* inst, int32_t n_inst, const float* mats, int32_t nm,
                              const float* camera, int32_t width, int32_t height) {
  const char* fn = "dr_scene_upload_instanced";
  if (!c || !meshes || !inst || !mats || !camera) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": NULL argument");
  if (n_meshes < 1 || n_inst < 1 || nm < 1) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": bad size");
  bool any_normals = false;
  for (int m = 0; m < n_meshes; ++m) {
    const dr_mesh_desc& q = meshes[m];
    if (!q.verts || !q.tris || !q.tri_mat || q.nv < 1 || q.nt < 1)
      return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": mesh " + std::to_string(m) + " is empty or NULL");
    for (long long k = 0; k < 3ll * q.nt; ++k)
      if (q.tris[k] < 0 || q.tris[k] >= q.nv)
        return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": mesh vertex index out of range");
    for (int k = 0; k < q.nt; ++k)
      if (q.tri_mat[k] < 0 || q.tri_mat[k] >= nm)
        return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": mesh material out of range");
    for (long long k = 0; k < 3ll * q.nv; ++k)
      if (!std::isfinite(q.verts[k])) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": non-finite vertex");
    any_normals = any_normals || q.normals != nullptr;
  }
  long long tv = 0, tt = 0;
  std::vector<double> inv(12 * (size_t)n_inst);
  for (int i = 0; i < n_inst; ++i) {
    const dr_instance_desc& d = inst[i];
    if (d.mesh < 0 || d.mesh >= n_meshes) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": instance mesh out of range");
    if (d.material < -1 || d.material >= nm)
      return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": instance material out of range");
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(d.xform[k])) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": non-finite transform");
    // inverse of A by cofactors over the determinant; c = -A^-1 t
    const double a00 = d.xform[0], a01 = d.xform[1], a02 = d.xform[2];
    const double a10 = d.xform[4], a11 = d.xform[5], a12 = d.xform[6];
    const double a20 = d.xform[8], a21 = d.xform[9], a22 = d.xform[10];
    const double c00 = a11 * a22 - a12 * a21, c01 = a12 * a20 - a10 * a22, c02 = a10 * a21 - a11 * a20;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det))
      return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": singular transform");
    double* M = inv.data() + 12 * (size_t)i;
    const double m[3][3] = {{c00 / det, (a02 * a21 - a01 * a22) / det, (a01 * a12 - a02 * a11) / det},
                            {c01 / det, (a00 * a22 - a02 * a20) / det, (a02 * a10 - a00 * a12) / det},
                            {c02 / det, (a01 * a20 - a00 * a21) / det, (a00 * a11 - a01 * a10) / det}};
    const double t[3] = {d.xform[3], d.xform[7], d.xform[11]};
    for (int row = 0; row < 3; ++row) {
      M[4 * row] = m[row][0];
      M[4 * row + 1] = m[row][1];
      M[4 * row + 2] = m[row][2];
      M[4 * row + 3] = -((m[row][0] * t[0] + m[row][1] * t[1]) + m[row][2] * t[2]);
    }
    tv += meshes[d.mesh].nv;
    tt += meshes[d.mesh].nt;
  }
  if (tv >= (1ll << 31) || tt >= (1ll << 30)) return fail(DR_ERR_INVALID_ARG, std::string(fn) + ": scene too large");
  // the flattened scene
  std::vector<float> V(3 * (size_t)tv), N(any_normals ? 3 * (size_t)tv : 0, 0.f), box(6 * (size_t)n_inst);
  std::vector<int> T(3 * (size_t)tt), TM((size_t)tt), tri_base(n_inst);
  std::vector<long long> vbase(n_inst);
  {
    long long vb = 0, tb = 0;
    for (int i = 0; i < n_inst; ++i) {
      vbase[i] = vb;
      tri_base[i] = (int)tb;
      vb += meshes[inst[i].mesh].nv;
      tb += meshes[inst[i].mesh].nt;
    }
  }
  // instances in parallel (disjoint output ranges)
  parallel_items(n_inst, [&](int i) {
    {
      const dr_instance_desc& d = inst[i];
      const dr_mesh_desc& q = meshes[d.mesh];
      const double* M = inv.data() + 12 * (size_t)i;
      const long long vb = vbase[i], tb = tri_base[i];
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int v = 0; v < q.nv; ++v) {
        const double p[3] = {q.verts[3 * v], q.verts[3 * v + 1], q.verts[3 * v + 2]};
        for (int row = 0; row < 3; ++row) {
          const double w = (((double)d.xform[4 * row] * p[0] + (double)d.xform[4 * row + 1] * p[1]) +
                            (double)d.xform[4 * row + 2] * p[2]) + (double)d.xform[4 * row + 3];
          const float f = (float)w;
          V[3 * (vb + v) + row] = f;
          lo[row] = std::min(lo[row], f);
          hi[row] = std::max(hi[row], f);
        }
        if (q.normals) {
          const double n[3] = {q.normals[3 * v], q.normals[3 * v + 1], q.normals[3 * v + 2]};
          for (int row = 0; row < 3; ++row)
            N[3 * (vb + v) + row] = (float)((M[row] * n[0] + M[4 + row] * n[1]) + M[8 + row] * n[2]);
        }
      }
      for (int k = 0; k < q.nt; ++k) {
        for (int e = 0; e < 3; ++e) T[3 * (tb + k) + e] = (int)(vb + q.tris[3 * k + e]);
        TM[tb + k] = d.material >= 0 ? d.material : q.tri_mat[k];
      }
      for (int a = 0; a < 3; ++a) {
        box[6 * i + a] = lo[a];
        box[6 * i + 3 + a] = hi[a];
      }
    }
  });
  int r = dr_scene_upload(c, V.data(), (int32_t)tv, T.data(), any_normals ? N.data() : nullptr, (int32_t)tt, TM.data(),
                          mats, nm, camera, width, height);
  if (r != DR_OK) return r;
  if (n_inst >= 2 && c->two_level) r = build_two_level(c, meshes, n_meshes, inst, n_inst, inv, tri_base, box);
  if (r != DR_OK) c->target = -1;
  return r;
}

int dr_two_level_info(dr_ctx* c, int32_t* n_instances, int32_t* n_tlas_nodes, int32_t* n_blas_nodes) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_two_level_info: NULL ctx");
  if (c->target != 0 || !c->tl_nodes) return fail(DR_ERR_STATE, "dr_two_level_info: no two-level BVH");
  if (n_instances) *n_instances = c->n_insts;
  if (n_tlas_nodes) *n_tlas_nodes = c->n_tl_nodes;
  if (n_blas_nodes) *n_blas_nodes = c->n_bl_nodes;
  return DR_OK;
}

int dr_bvh4_sah(dr_ctx* c, double* node_steps, double* tri_tests) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_bvh4_sah: NULL ctx");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_bvh4_sah: no scene");
  if (!c->nodes4) return fail(DR_ERR_STATE, "dr_bvh4_sah: the scene has no 4-wide BVH");
  if (node_steps) *node_steps = c->bvh4_sah_nodes;
  if (tri_tests) *tri_tests = c->bvh4_sah_tris;
  return DR_OK;
}

int dr_bvh8_info(dr_ctx* c, int32_t* n_nodes, int32_t* max_depth) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_bvh8_info: NULL ctx");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_bvh8_info: no scene");
  if (!c->nodes8) return fail(DR_ERR_STATE, "dr_bvh8_info: the scene has no 8-wide BVH");
  if (n_nodes) *n_nodes = c->n_nodes8;
  if (max_depth) *max_depth = c->bvh8_depth;
  return DR_OK;
}

int dr_bvh_info(dr_ctx* c, int32_t* n_nodes, int32_t* n_tris, int32_t* max_depth) {
  if (!c) return fail(DR_ERR_INVALID_ARG, "dr_bvh_info: NULL ctx");
  if (c->target != 0) return fail(DR_ERR_STATE, "dr_bvh_info: no scene");
  DR_CUDA(cudaSetDevice(c->device));
  const int nn = std::max(1, c->n_nodes);
  std::vector<float4> nodes((size_t)nn * 4);
  DR_CUDA(cudaMemcpyAsync(nodes.data(), c->nodes, nodes.size() * 16, cudaMemcpyDeviceToHost, c->stream));
  DR_CUDA(cudaStreamSynchronize(c->stream));
  // walk the hierarchy once, checking that it is a tree: every inner node is
  // reached exactly once and every triangle lies in exactly one leaf
  int depth = 0;
  std::vector<uint8_t> seen_node((size_t)nn, 0), seen_tri((size_t)std::max(1, c->nt), 0);
  std::vector<std::pair<int, int>> st{{0, 1}};
  long long leaves_tris = 0;
  while (!st.empty()) {
    auto [n, dd] = st.back();
    st.pop_back();
    if (n < 0 || n >= nn) return fail(DR_ERR_DEVICE_CHECK, "dr_bvh_info: corrupt node index");
    if (seen_node[n]++) return fail(DR_ERR_DEVICE_CHECK, "dr_bvh_info: node reached twice (not a tree)");
    depth = std::max(depth, dd);
    const int ch[2] = {hbits_i(nodes[4 * n + 3].x), hbits_i(nodes[4 * n + 3].y)};
    for (int k = 0; k < 2; ++k) {
      if (ch[k] >= 0) {
        st.push_back({ch[k], dd + 1});
      } else if (!(c->nt == 1 && k == 1)) {  // a one-triangle scene repeats its leaf
        const int first = leaf_first(ch[k]), cnt = leaf_count(ch[k]);
        for (int i = first; i < first + cnt; ++i) {
          if (i >= c->nt || seen_tri[i]++) return fail(DR_ERR_DEVICE_CHECK, "dr_bvh_info: bad or repeated leaf");
          ++leaves_tris;
        }
      }
    }
  }
  if (leaves_tris != c->nt) return fail(DR_ERR_DEVICE_CHECK, "dr_bvh_info: triangles missing from the leaves");
  for (int i = 0; i < c->n_nodes; ++i)
    if (!seen_node[i]) return fail(DR_ERR_DEVICE_CHECK, "dr_bvh_info: unreachable inner node");
  if (n_nodes) *n_nodes = c->n_nodes;
  if (n_tris) *n_tris = c->nt;
  if (max_depth) *max_depth = depth;
  return DR_OK;
}

}  // extern "C"
