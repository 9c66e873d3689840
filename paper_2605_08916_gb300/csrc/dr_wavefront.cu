// Wavefront execution of one Restore step with the adjoint drift: instead
// of one thread tracing a whole path (plus NEE and the reverse sweep), each
// bounce is a separate pass over a compacted queue of the paths still alive:
//
//   wf_begin      Evolve (regenerate / LocalDynamics) and the camera ray
//   per bounce k  wf_trace   closest hit of every queued ray
//                 wf_shade   path_vertex: tape entry, emission, NEE request,
//                            BSDF sample; survivors go to the next queue,
//                            NEE requests to the shadow queue
//                 wf_shadow  any-hit test of each NEE ray, contribution add
//   wf_finish     p = lum(f) + eps, hold/kill clock, splat record; chains
//                 that survive go to the adjoint queue
//   wf_adjoint    reverse sweep over the tape kept in HBM
//
// Queues are compacted with ballots and popcounts and one atomic per block
// iteration (shading) or per warp (the rest), so warps never carry finished
// paths; the traversal passes are small kernels
// with few registers.  Every path accumulates its contributions in the same
// order as the fused kernel (emission of hit k, NEE of vertex k, emission of
// hit k + 1, ...); the two executions differ only where the compiler
// contracts multiply-adds differently (last-bit differences).
#include "dr_step.cuh"

namespace dr {

namespace {

constexpr int kWfThreads = 128;
constexpr int kWfStack = kTraversalStack;
// stack entries of the persistent passes per walk
constexpr int wf_stack(int width) { return width == kWalkTwoLevel ? kTraversalStackTL : kWfStack; }
// (the two-level traversal's larger stack leaves room for 6 blocks per SM,
// so it is compiled for 6 and may use more registers)
// resident blocks per SM the traversal passes are compiled for (register cap)
constexpr int kWfTraceMinBlocks = 10;
// the 4-wide traversal holds four child boxes at once: fewer resident
// blocks, more registers per thread (measured: 7 beats 6 and 8)
constexpr int kWfTrace4MinBlocks = 7;
// shading waits on its loads: more resident warps (80 registers) hide more
// (measured: 6 blocks beat 5 on the 1M-triangle and batch workloads)
constexpr int kWfShadeMinBlocks = 6;

// 64-B path slot per chain: (o, ppdf), (d, prev tri), (beta, prev_delta |
// nseg << 8), (f, pixel)
DR_D void load_slot(const float4* __restrict__ slot, unsigned long long j, PathState& ps, int& pix) {
  const float4 a = slot[4 * j + 0], b = slot[4 * j + 1], c = slot[4 * j + 2], d = slot[4 * j + 3];
  ps.o = xyz(a);
  ps.ppdf = a.w;
  ps.d = xyz(b);
  ps.prev_tri = __float_as_int(b.w);
  ps.beta = xyz(c);
  const int fl = __float_as_int(c.w);
  ps.prev_delta = fl & 1;
  ps.nseg = fl >> 8;
  ps.f = xyz(d);
  pix = __float_as_int(d.w);
}

DR_D void store_slot(float4* __restrict__ slot, unsigned long long j, const PathState& ps, int pix) {
  slot[4 * j + 0] = make_float4(ps.o.x, ps.o.y, ps.o.z, ps.ppdf);
  slot[4 * j + 1] = make_float4(ps.d.x, ps.d.y, ps.d.z, __int_as_float(ps.prev_tri));
  slot[4 * j + 2] = make_float4(ps.beta.x, ps.beta.y, ps.beta.z, __int_as_float((ps.prev_delta & 1) | (ps.nseg << 8)));
  slot[4 * j + 3] = make_float4(ps.f.x, ps.f.y, ps.f.z, __int_as_float(pix));
}

// Appends to one of several queues (counters[key]): the lanes of `want`
// (every lane calling, and only those) group by key, one atomic per group.
DR_D uint32_t keyed_append(uint32_t* counters, int key, unsigned want) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(want, key);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&counters[key], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// Ray queue of bounce k (the two queues alternate).  Selected with a
// branch, not an index: a run-time index into the kernel-parameter struct
// would make the compiler copy the whole struct to local memory.
DR_D uint32_t* queue_of(const WfBuffers& w, int k) { return (k & 1) ? w.queue[1] : w.queue[0]; }

DR_D void add_counts(unsigned long long* target, unsigned long long v) {
  const unsigned long long w = warp_sum_u64(v);
  if ((threadIdx.x & 31) == 0 && w && target) atomicAdd(target, w);
}

// Per-chain view of the target: the single scene, or in a multi-scene batch
// the chain's own scene (index sid, path length, PSS dimension, first pixel
// in the shared image).  A batch chain draws Philox numbers with its index
// within its scene and the key (seed_lo, seed_hi + sid), so each scene of a
// batch evolves exactly as it would in a context of its own.
struct ChainView {
  int sid, L, d;
  uint32_t cj, pix0;
};

template <bool BATCH>
DR_D ChainView chain_view(const StepArgs& a, unsigned long long j) {
  if (!BATCH) return ChainView{0, a.L, a.d, (uint32_t)j, 0u};
  const int s = a.chain_scene[j];
  const SceneChains& sc = a.sc[s];
  return ChainView{s, sc.L, sc.d, (uint32_t)(j - sc.chain0), sc.pix0};
}

template <bool BATCH>
DR_D Rng chain_rng(const StepArgs& a, const ChainView& v) {
  Rng r = rng_of(a);
  if (BATCH) r.k1 += (uint32_t)v.sid;
  return r;
}

template <bool BATCH>
DR_D const DevScene& scene_of(const StepArgs& a, int sid) {
  return BATCH ? a.scenes[sid] : a.S;
}

// Morton (Z-order) interleave of two 16-bit coordinates
DR_D uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
DR_D uint32_t morton2(uint32_t x, uint32_t y) { return spread16(x) | (spread16(y) << 1); }

// queue[1] = the chains of the sorted (key, chain) pairs
__global__ void wf_order_queue(const uint2* __restrict__ sorted, unsigned long long n, uint32_t* __restrict__ q) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) q[t] = sorted[t].y;
}

template <bool BATCH>
__global__ void __launch_bounds__(kWfThreads) wf_begin(StepArgs a, WfBuffers w) {
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < a.N;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    const ChainView v = chain_view<BATCH>(a, j);
    evolve_x(a, chain_rng<BATCH>(a, v), step_index(a), j, v.cj, v.d, a.init || a.killed[j] != 0);
    PathState ps;
    const DevScene& S = scene_of<BATCH>(a, v.sid);
    const int pix = path_begin(S, XSoA{a.x, a.N, j}, ps);
    if (a.ray_keys) {
      const uint32_t px = (uint32_t)pix % (uint32_t)S.W, py = (uint32_t)pix / (uint32_t)S.W;
      uint32_t key = morton2(px, py);
      if (BATCH) key |= (uint32_t)v.sid << a.key_shift;
      a.ray_keys[j] = make_uint2(key, (uint32_t)j);
    }
    store_slot(w.slot, j, ps, pix);
    w.hit[j] = -1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) w.counts[1] = (uint32_t)a.N;  // bounce 1: every chain
}

// binary-BVH trace pass: one closest-hit ray per thread, grid-stride
template <bool STATS>
__global__ void __launch_bounds__(kWfThreads, kWfTraceMinBlocks) wf_trace(StepArgs a, WfBuffers w, int k) {
  extern __shared__ int smem[];
  TraceStack<kWfStack> st{smem + threadIdx.x, (int)blockDim.x};
  const uint32_t n = w.counts[k];
  const uint32_t* q = k == 1 && !a.ray_keys ? nullptr : queue_of(w, k);
  uint32_t err = 0;
  TraceStats stats{0u, 0u};
  unsigned long long rays = 0;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const unsigned long long j = q ? q[t] : t;
    const float4 o = w.slot[4 * j + 0], d = w.slot[4 * j + 1];
    float th;
    w.hit[j] = trace_closest<kWfStack, STATS, 2>(a.S, make_ray(xyz(o), xyz(d)), __float_as_int(d.w), &th, st,
                                                     &err, &stats);
    ++rays;
  }
  add_counts(a.rays, rays);
  if (STATS) {
    add_counts(a.node_visits, stats.nodes);
    add_counts(a.tri_tests, stats.tris);
  }
  if (err) atomicOr(a.err, err);
}

// Persistent 4-wide trace passes with dynamic ray fetch: a warp keeps
// stepping its lanes' walks one node at a time and, whenever fewer than
// a.refill lanes (16 of 32 by default; with inner-node and leaf steps
// alternated by majority, measured better than 20-32)
// still hold a ray, refills the idle lanes from the queue with one atomic
// per warp.  A warp's time is then set by its total work
// rather than by its slowest ray.
constexpr unsigned kFull = 0xffffffffu;

// Hands the idle lanes of a warp (mask `idle`) consecutive queue positions;
// returns this lane's position (valid for idle lanes) and whether the queue
// of n entries is now drained.  All 32 lanes call it together.
DR_D uint32_t warp_fetch(uint32_t* ctr, unsigned idle, uint32_t n, bool& drained) {
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(idle) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(ctr, (uint32_t)__popc(idle));
  base = __shfl_sync(kFull, base, leader);
  if (base + (uint32_t)__popc(idle) >= n) drained = true;
  return base + __popc(idle & ((1u << lane) - 1u));
}

// One traversal pass of the 4-wide path: the closest-hit rays of bounce k
// (n_ray of them; none when k > L) and the shadow rays of bounce k - 1
// (n_shadow; none when k = 1) share one fetch counter, closest-hit rays
// first.  The two sets touch disjoint data (hit[] and the ray state vs. the
// path's f and the shadow-visibility tape flag), so one launch replaces two
// and each bounce pays the latency of its slowest ray once.
template <bool STATS, bool BATCH, int WIDTH>
__global__ void __launch_bounds__(kWfThreads, WIDTH == kWalkTwoLevel ? 6 : kWfTrace4MinBlocks)
    wf_traverse(StepArgs a, WfBuffers w, int k) {
  extern __shared__ int smem[];
  constexpr int kS = wf_stack(WIDTH);
  TraceStack<kS> st{smem + threadIdx.x, (int)blockDim.x};
  const uint32_t n_ray = k <= a.L ? w.counts[k] : 0u;
  const uint32_t n_shadow = k >= 2 ? w.counts[kWfShadowCount0 + k - 1] : 0u;
  const uint32_t n = n_ray + n_shadow;
  const uint32_t* q = k == 1 && !a.ray_keys ? nullptr : queue_of(w, k);
  uint32_t* ctr = &w.counts[kWfFetch0 + k];
  uint32_t err = 0;
  TraceStats stats{0u, 0u};
  unsigned long long rays = 0;
  bool has = false, drained = false, shadow = false;
  uint32_t j = 0, t = 0;
  int ex0 = -1, ex1 = -1, best = -1, sid = 0;
  float tlim = 0.0f;  // closest hit so far, or the shadow ray's tmax
  Ray r;
  typename WalkOf<WIDTH>::type wk{};
  // a pass with few rays (the late bounces) spreads them over every warp of
  // the grid: a warp then walks a few rays, and the pass, which lasts as
  // long as its slowest warp, ends sooner
  const uint32_t n_warps = gridDim.x * (blockDim.x / 32u);
  const int cap = (int)min(32u, max(1u, (n + n_warps - 1u) / n_warps));
  const int refill = cap >= 32 ? a.refill : max(1, cap / 2);
  const int lane = threadIdx.x & 31;
  while (true) {
    if (!drained) {
      const unsigned idle = __ballot_sync(kFull, !has);
      // the idle lanes that take a ray: the lowest ones, up to cap busy lanes
      unsigned take = idle;
      const int room = cap - (32 - __popc(idle));
      if (room < __popc(idle)) {
        unsigned m = idle;
        take = 0u;
        for (int i = 0; i < room; ++i) {
          const unsigned low = m & (0u - m);
          take |= low;
          m ^= low;
        }
      }
      if (take) {
        const uint32_t tn = warp_fetch(ctr, take, n, drained);
        if (((take >> lane) & 1u) && tn < n) {
          shadow = tn >= n_ray;
          if (shadow) {
            t = tn - n_ray;
            const ShadowRec& sr = w.shadow[t];
            const float4 o = sr.o_tmax, d = sr.wi_chain;
            r = make_ray(xyz(o), xyz(d));
            tlim = o.w;
            ex0 = __float_as_int(sr.contrib_ex.w);
            ex1 = sr.ex1;
            if (BATCH) sid = a.chain_scene[__float_as_int(d.w)];
          } else {
            j = q ? q[tn] : tn;
            const float4 o = w.slot[4 * (size_t)j + 0], d = w.slot[4 * (size_t)j + 1];
            r = make_ray(xyz(o), xyz(d));
            ex0 = __float_as_int(d.w);
            tlim = __int_as_float(0x7f800000);
            best = -1;
            if (BATCH) sid = a.chain_scene[j];
          }
          walk_begin(scene_of<BATCH>(a, sid), r, wk);
          ++rays;
          if (ray_finite(r.o, r.d)) {
            has = true;
          } else {
            err |= kErrNonFinite;  // no hit; a shadow ray counts as occluded
            if (!shadow) w.hit[j] = -1;
          }
        }
      }
    }
    if (__ballot_sync(kFull, has) == 0) {
      if (drained) break;
      continue;
    }
    while (true) {
      // inner-node steps and leaf steps are different code: a warp takes
      // the kind that more of its lanes are at, and the other lanes wait a
      // step, so each kind runs with many lanes at once
      const bool lf = walk_at_leaf(wk);
      const unsigned at_leaf = __ballot_sync(kFull, has && lf);
      const unsigned at_inner = __ballot_sync(kFull, has && !lf);
      const bool leaf_phase = __popc(at_leaf) >= __popc(at_inner);
      if (has && lf == leaf_phase) {
        const DevScene& S = scene_of<BATCH>(a, sid);
        bool done, occ = false;
        if constexpr (WIDTH == 4) {
          // closest-hit and shadow rays share one step (one instruction
          // stream for a warp that holds both)
          done = mixed4_step<kS, STATS>(S, r, shadow, ex0, shadow ? ex1 : -1, wk, tlim, best, &occ, st, &err, &stats);
        } else {
          done = !shadow ? closest_step<kS, STATS>(S, r, ex0, wk, tlim, best, st, &err, &stats)
                         : any_step<kS, STATS>(S, r, tlim, ex0, ex1, wk, &occ, st, &err, &stats);
        }
        if (done) {
          has = false;
          if (!shadow) {
            w.hit[j] = best;
          } else {
            if (!occ) {
              const ShadowRec& sr = w.shadow[t];
              const unsigned long long c = (unsigned long long)__float_as_int(sr.wi_chain.w);
              float4 f = w.slot[4 * c + 3];
              f.x += sr.contrib_ex.x;
              f.y += sr.contrib_ex.y;
              f.z += sr.contrib_ex.z;
              w.slot[4 * c + 3] = f;
              GlobalTape{w.tape, a.N, c}.or_flags(k - 2, kFNeeVis);
            }
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, has);
      if (act == 0 || (!drained && __popc(act) < refill)) break;
    }
  }
  add_counts(a.rays, rays);
  if (STATS) {
    add_counts(a.node_visits, stats.nodes);
    add_counts(a.tri_tests, stats.tris);
  }
  if (err) atomicOr(a.err, err);
}

template <bool BATCH, bool COND>
__global__ void __launch_bounds__(kWfThreads, kWfShadeMinBlocks) wf_shade(StepArgs a, WfBuffers w, int k) {
  const uint32_t n = w.counts[k];
  const uint32_t* q = k == 1 && !a.ray_keys ? nullptr : queue_of(w, k);
  uint32_t* qn = queue_of(w, k + 1);
  const uint32_t n_iter = (n + gridDim.x * blockDim.x - 1) / (gridDim.x * blockDim.x);
  // the queue appends are aggregated over the block: one atomic per counter
  // and block iteration instead of one per warp, since atomics on one address
  // serialise (measured: shading 0.31 -> 0.26 ms per caustic step); the
  // per-warp counts are double-buffered by iteration parity
  __shared__ uint32_t s_cnt[2][2][kWfThreads / 32];
  __shared__ uint32_t s_base[2][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // every thread runs the same number of iterations so the queue appends see
  // whole warps and the whole block
  for (uint32_t it = 0; it < n_iter; ++it) {
    const uint32_t t = it * gridDim.x * blockDim.x + blockIdx.x * blockDim.x + threadIdx.x;
    bool cont = false;
    NeeReq nee;
    nee.valid = false;
    unsigned long long j = 0;
    int L = a.L;
    if (t < n) {
      j = q ? q[t] : t;
      const int tri = w.hit[j];
      const ChainView v = chain_view<BATCH>(a, j);
      L = v.L;
      if (tri >= 0) {
        PathState ps;
        int pix;
        load_slot(w.slot, j, ps, pix);
        cont = path_vertex<COND>(scene_of<BATCH>(a, v.sid), XSoA{a.x, a.N, j}, L, k, tri, ps, GlobalTape{w.tape, a.N, j},
                           nee);
        store_slot(w.slot, j, ps, pix);
      }
    }
    const bool next = cont && k < L;
    const int par = it & 1;
    const unsigned ms = __ballot_sync(kFull, nee.valid), mn = __ballot_sync(kFull, next);
    if (lane == 0) {
      s_cnt[par][0][wid] = __popc(ms);
      s_cnt[par][1][wid] = __popc(mn);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      uint32_t tot = 0;
      for (int q2 = 0; q2 < kWfThreads / 32; ++q2) tot += s_cnt[par][threadIdx.x][q2];
      s_base[par][threadIdx.x] =
          tot ? atomicAdd(&w.counts[threadIdx.x == 0 ? kWfShadowCount0 + k : k + 1], tot) : 0u;
    }
    __syncthreads();
    uint32_t ws = s_base[par][0], wn = s_base[par][1];
    for (int q2 = 0; q2 < wid; ++q2) {
      ws += s_cnt[par][0][q2];
      wn += s_cnt[par][1][q2];
    }
    const unsigned below = (1u << lane) - 1u;
    const uint32_t si = ws + __popc(ms & below), ni = wn + __popc(mn & below);
    if (nee.valid) {
      ShadowRec r;
      r.o_tmax = make_float4(nee.o.x, nee.o.y, nee.o.z, nee.tmax);
      r.wi_chain = make_float4(nee.wi.x, nee.wi.y, nee.wi.z, __int_as_float((int)j));
      r.contrib_ex = make_float4(nee.contrib.x, nee.contrib.y, nee.contrib.z, __int_as_float(nee.ex0));
      r.ex1 = nee.ex1;
      w.shadow[si] = r;
    }
    if (next) {
      qn[ni] = (uint32_t)j;
      w.hit[j] = -1;
    }
  }
}

// The tail of a step in one persistent pass: from the shading of bounce k0
// on, each lane carries a whole path (shade, its shadow ray, the next
// closest-hit ray, shade, ...) until it ends, and fetches another path from
// the bounce-k0 queue whenever fewer than a.refill lanes are busy.  Late
// bounces have few rays, so separate launches per bounce would each wait for
// their slowest ray; here those waits overlap.  The per-path order of work,
// and with it every addition to f and every tape write, is the one of the
// bounce-by-bounce passes, so the results are identical.
constexpr int kWfTailMinBlocks = 4;

template <bool STATS, bool BATCH, bool COND, int WIDTH>
__global__ void __launch_bounds__(kWfThreads, kWfTailMinBlocks) wf_tail(StepArgs a, WfBuffers w, int k0) {
  extern __shared__ int smem[];
  constexpr int kS = wf_stack(WIDTH);
  TraceStack<kS> st{smem + threadIdx.x, (int)blockDim.x};
  enum { kIdle = 0, kShade, kClosest, kShadow };
  const uint32_t n = w.counts[k0];
  const uint32_t* q = k0 == 1 && !a.ray_keys ? nullptr : queue_of(w, k0);
  uint32_t* ctr = &w.counts[kWfFetch0 + 0];  // the fetch counter of bounce 0 is otherwise unused
  uint32_t err = 0;
  TraceStats stats{0u, 0u};
  unsigned long long rays = 0;
  bool drained = false, cont_after = false;
  int state = kIdle, k = 0, hit = -1, L = a.L, sid = 0, ex0 = -1, ex1 = -1, best = -1;
  unsigned long long j = 0;
  PathState ps;
  int pix = 0;
  Ray r;
  typename WalkOf<WIDTH>::type wk{};
  float tlim = 0.0f;
  float3 contrib = f3(0.f, 0.f, 0.f);
  while (true) {
    if (!drained) {
      const unsigned idle = __ballot_sync(kFull, state == kIdle);
      if (idle) {
        const uint32_t t = warp_fetch(ctr, idle, n, drained);
        if (state == kIdle && t < n) {
          j = q ? q[t] : t;
          load_slot(w.slot, j, ps, pix);
          hit = w.hit[j];
          const ChainView v = chain_view<BATCH>(a, j);
          L = v.L;
          sid = v.sid;
          k = k0;
          state = kShade;
        }
      }
    }
    if (__ballot_sync(kFull, state != kIdle) == 0) {
      if (drained) break;
      continue;
    }
    while (true) {
      const DevScene& S = scene_of<BATCH>(a, sid);
      // shading is long and walking steps are short: a warp shades only
      // when at least as many of its lanes wait to shade as walk, so the
      // shading runs with many lanes at once
      const unsigned shading = __ballot_sync(kFull, state == kShade);
      const unsigned walking = __ballot_sync(kFull, state == kClosest || state == kShadow);
      const bool do_shade = __popc(shading) >= __popc(walking);
      if (state == kShade && do_shade) {
        bool next = false;
        if (hit >= 0) {
          NeeReq nee;
          nee.valid = false;
          const bool cont = path_vertex<COND>(S, XSoA{a.x, a.N, j}, L, k, hit, ps, GlobalTape{w.tape, a.N, j}, nee);
          next = cont && k < L;
          if (nee.valid) {
            r = make_ray(nee.o, nee.wi);
            tlim = nee.tmax;
            ex0 = nee.ex0;
            ex1 = nee.ex1;
            contrib = nee.contrib;
            cont_after = next;
            walk_begin(S, r, wk);
            ++rays;
            if (ray_finite(r.o, r.d)) {
              state = kShadow;
            } else {
              err |= kErrNonFinite;  // occluded: no contribution
            }
          }
        }
        if (state == kShade) {  // no shadow ray to walk
          if (next) {
            ++k;
            r = make_ray(ps.o, ps.d);
            ex0 = ps.prev_tri;
            tlim = __int_as_float(0x7f800000);
            best = -1;
            walk_begin(S, r, wk);
            ++rays;
            if (ray_finite(r.o, r.d)) {
              state = kClosest;
            } else {
              err |= kErrNonFinite;
              hit = -1;  // shaded as a miss
            }
          } else {
            store_slot(w.slot, j, ps, pix);
            state = kIdle;
          }
        }
      } else if ((state == kShadow || state == kClosest) && !do_shade) {
        // closest-hit and shadow walks share one step (one instruction
        // stream for a warp that holds both)
        const bool sh = state == kShadow;
        bool done, occ = false;
        if constexpr (WIDTH == 4) {
          done = mixed4_step<kS, STATS>(S, r, sh, ex0, sh ? ex1 : -1, wk, tlim, best, &occ, st, &err, &stats);
        } else {
          done = sh ? any_step<kS, STATS>(S, r, tlim, ex0, ex1, wk, &occ, st, &err, &stats)
                    : closest_step<kS, STATS>(S, r, ex0, wk, tlim, best, st, &err, &stats);
        }
        if (done && !sh) {
          hit = best;
          state = kShade;
        } else if (done) {
          if (!occ) {
            ps.f += contrib;
            GlobalTape{w.tape, a.N, j}.or_flags(k - 1, kFNeeVis);
          }
          if (cont_after) {
            ++k;
            r = make_ray(ps.o, ps.d);
            ex0 = ps.prev_tri;
            tlim = __int_as_float(0x7f800000);
            best = -1;
            walk_begin(S, r, wk);
            ++rays;
            if (ray_finite(r.o, r.d)) {
              state = kClosest;
            } else {
              err |= kErrNonFinite;
              hit = -1;
              state = kShade;
            }
          } else {
            store_slot(w.slot, j, ps, pix);
            state = kIdle;
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, state != kIdle);
      if (act == 0 || (!drained && __popc(act) < a.refill)) break;
    }
  }
  add_counts(a.rays, rays);
  if (STATS) {
    add_counts(a.node_visits, stats.nodes);
    add_counts(a.tri_tests, stats.tris);
  }
  if (err) atomicOr(a.err, err);
}

// binary-BVH shadow pass of bounce k
template <bool STATS>
__global__ void __launch_bounds__(kWfThreads, kWfTraceMinBlocks) wf_shadow(StepArgs a, WfBuffers w, int k) {
  extern __shared__ int smem[];
  TraceStack<kWfStack> st{smem + threadIdx.x, (int)blockDim.x};
  const uint32_t n = w.counts[kWfShadowCount0 + k];
  uint32_t err = 0;
  TraceStats stats{0u, 0u};
  unsigned long long rays = 0;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const ShadowRec r = w.shadow[t];
    const unsigned long long j = (unsigned long long)__float_as_int(r.wi_chain.w);
    ++rays;
    if (!trace_any<kWfStack, STATS, 2>(a.S, make_ray(xyz(r.o_tmax), xyz(r.wi_chain)), r.o_tmax.w,
                                           __float_as_int(r.contrib_ex.w), r.ex1, st, &err, &stats)) {
      float4 f = w.slot[4 * j + 3];
      f.x += r.contrib_ex.x;
      f.y += r.contrib_ex.y;
      f.z += r.contrib_ex.z;
      w.slot[4 * j + 3] = f;
      GlobalTape{w.tape, a.N, j}.or_flags(k - 1, kFNeeVis);
    }
  }
  add_counts(a.rays, rays);
  if (STATS) {
    add_counts(a.node_visits, stats.nodes);
    add_counts(a.tri_tests, stats.tris);
  }
  if (err) atomicOr(a.err, err);
}

// Accumulate: the kill clock, the state written back and the splat record
// (mode kWfStep / kWfInitClock); the chains that survive go to the adjoint
// queue (kWfStep).  kWfInitEval instead stores p and queues every chain.
template <bool BATCH>
__global__ void __launch_bounds__(kWfThreads) wf_finish(StepArgs a, WfBuffers w, int mode, float* p_out) {
  const unsigned long long n_iter = (a.N + (unsigned long long)gridDim.x * blockDim.x - 1) /
                                    ((unsigned long long)gridDim.x * blockDim.x);
  uint32_t err = 0;
  unsigned long long kills = 0;
  for (unsigned long long it = 0; it < n_iter; ++it) {
    const unsigned long long j = it * gridDim.x * blockDim.x + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool survive = false;
    int nseg = 0;
    int kill_sid = -1;  // batch: the scene of a chain killed here
    if (j < a.N) {
      PathState ps;
      int pix;
      load_slot(w.slot, j, ps, pix);
      nseg = min(max(ps.nseg, 0), kMaxPathLen);
      const float3 f = ps.f;
      const float p = lum(f) + a.eps;
      if (!(isfinite(p) && isfinite(f.x) && isfinite(f.y) && isfinite(f.z))) err |= kErrNonFinite;
      if (a.plen) a.plen[j] = (uint8_t)ps.nseg;
      if (mode == kWfInitEval) {
        p_out[j] = p;
        survive = a.drift != 0;  // without a drift no score is computed
      } else {
        const ChainView v = chain_view<BATCH>(a, j);
        const U4 rc = chain_rng<BATCH>(a, v).draw(step_index(a), v.cj, 0u, kClock);
        bool killed;
        float wt;
        kill_clock(a.rb, u01(rc.a), u01(rc.b), p, a.h, BATCH ? a.sc[v.sid].k0 : k0_of(a), &killed, &wt);
        a.killed[j] = killed ? 1 : 0;
        a.logp[j] = logf(p);
        if (BATCH) {
          if (killed) kill_sid = v.sid;
        } else {
          kills += killed ? 1ull : 0ull;
        }
        if (a.rec) {
          const float s = wt / p;
          SplatRec rr;
          rr.pix = v.pix0 + (uint32_t)pix;
          rr.r = f.x * s;
          rr.g = f.y * s;
          rr.b = f.z * s;
          a.rec[j] = rr;
        }
        survive = !killed && mode == kWfStep && a.drift != 0;
      }
    }
    // a batch's tour counts: one atomic per scene present among the warp's
    // killed chains (every lane runs the same number of iterations)
    if (BATCH) {
      const unsigned want = __ballot_sync(kFull, kill_sid >= 0);
      if (kill_sid >= 0) {
        const unsigned peers = __match_any_sync(want, kill_sid);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
          atomicAdd(a.sc[kill_sid].tour_count, (unsigned long long)__popc(peers));
      }
    }
    // survivors queue by path length, so that the adjoint's warps run
    // loops of equal trip count
    if (survive) {
      const uint32_t ai = keyed_append(&w.counts[kWfAdjBucket0], nseg, __ballot_sync(__activemask(), true));
      w.adj[(size_t)nseg * a.N + ai] = (uint32_t)j;
    }
  }
  add_counts(a.tour_count, kills);
  if (err) atomicOr(a.err, err);
}

template <bool BATCH, bool COND>
__global__ void __launch_bounds__(kWfThreads, 4) wf_adjoint(StepArgs a, WfBuffers w) {
  // the queue is the concatenation of the path-length buckets, longest first
  __shared__ uint32_t off[kMaxPathLen + 2];
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int b = kMaxPathLen; b >= 0; --b) {
      off[b + 1] = acc;
      acc += w.counts[kWfAdjBucket0 + b];
    }
    off[0] = acc;  // total
  }
  __syncthreads();
  const uint32_t n = off[0];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    int b = kMaxPathLen;
    while (b > 0 && t >= off[b]) --b;  // bucket b holds positions [off[b + 1], off[b])
    const unsigned long long j = w.adj[(size_t)b * a.N + (t - off[b + 1])];
    if (j >= a.N || t - off[b + 1] >= a.N) {
      atomicOr(a.err, kErrBadIndex);
      continue;
    }
    PathState ps;
    int pix;
    load_slot(w.slot, j, ps, pix);
    const float p = lum(ps.f) + a.eps;
    const ChainView v = chain_view<BATCH>(a, j);
    path_adjoint<COND>(scene_of<BATCH>(a, v.sid), XSoA{a.x, a.N, j}, v.L, p, GlobalTape{w.tape, a.N, j}, ps.nseg,
                 GSoA{a.score, a.N, j});
  }
}

unsigned grid_for(unsigned long long n, int max_blocks) {
  const unsigned long long b = (n + kWfThreads - 1) / kWfThreads;
  return (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>(b, (unsigned long long)max_blocks));
}

// resident blocks per SM of the persistent traversal pass, computed once
template <bool BATCH, int WIDTH>
int traverse_blocks_per_sm(size_t smem) {
  static int cached = 0;
  if (cached == 0) {
    int b0 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, wf_traverse<false, BATCH, WIDTH>, kWfThreads, smem);
    cached = std::max(1, b0);
  }
  return cached;
}

template <bool BATCH, bool COND, int WIDTH>
int tail_blocks_per_sm(size_t smem) {
  static int cached = 0;
  if (cached == 0) {
    int b0 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, wf_tail<false, BATCH, COND, WIDTH>, kWfThreads, smem);
    cached = std::max(1, b0);
  }
  return cached;
}

template <bool BATCH, bool COND, int WIDTH>
int launch_wf(const StepArgs& a, const WfBuffers& w, bool stats, int n_sm, const WfTuning& tune,
              const PhaseHook& hook, cudaStream_t s, WfMode mode, float* p_out, const RayOrder& order) {
  const int max_blocks = n_sm * 16;
  const unsigned g = grid_for(a.N, max_blocks);
  if (mode == kWfInitClock) {
    hook(kPhFinish, true);
    wf_finish<BATCH><<<g, kWfThreads, 0, s>>>(a, w, mode, p_out);
    hook(kPhFinish, false);
    return 1;
  }
  const size_t smem = (size_t)wf_stack(WIDTH) * kWfThreads * sizeof(int);
  const bool wide = a.S.nodes4 != nullptr || BATCH;
  // persistent traversal: as many blocks as stay resident (or fewer, tuned)
  const int resident = traverse_blocks_per_sm<BATCH, WIDTH>(smem);
  const int per_sm = tune.blocks_per_sm > 0 ? std::min(tune.blocks_per_sm, resident) : resident;
  const unsigned g4 = (unsigned)(n_sm * per_sm);
  int launches = 0;
  cudaMemsetAsync(w.counts, 0, kWfCounts * sizeof(uint32_t), s);
  hook(kPhBegin, true);
  wf_begin<BATCH><<<g, kWfThreads, 0, s>>>(a, w);
  hook(kPhBegin, false);
  launches += 2;
  if (a.ray_keys) {
    // camera rays in pixel (Morton) order: neighbouring lanes trace
    // neighbouring rays, here and, through the order-keeping queue
    // appends, at later bounces
    hook(kPhOrder, true);
    const uint2* sorted = sort_pairs(order.keys, order.alt, a.N, order.bits, order.scratch, s);
    wf_order_queue<<<(unsigned)((a.N + 255) / 256), 256, 0, s>>>(sorted, a.N, w.queue[1]);
    hook(kPhOrder, false);
    launches += 1 + 5 * ((order.bits + 7) / 8);
  }
  if (wide) {
    // traverse(k) = closest-hit rays of bounce k + shadow rays of bounce
    // k - 1; the last launch (k = L + 1) carries the final shadow rays
    for (int k = 1; k <= a.L + 1; ++k) {
      hook(k <= a.L ? kPhTrace : kPhShadow, true, k <= a.L ? k : a.L);
      if (stats) wf_traverse<true, BATCH, WIDTH><<<g4, kWfThreads, smem, s>>>(a, w, k);
      else wf_traverse<false, BATCH, WIDTH><<<g4, kWfThreads, smem, s>>>(a, w, k);
      hook(k <= a.L ? kPhTrace : kPhShadow, false, k <= a.L ? k : a.L);
      launches += 1;
      if (k <= a.L && k == tune.tail_bounce) {
        // the rest of every path in one persistent pass
        hook(kPhTail, true, k);
        const unsigned gt = (unsigned)(n_sm * tail_blocks_per_sm<BATCH, COND, WIDTH>(smem));
        if (stats) wf_tail<true, BATCH, COND, WIDTH><<<gt, kWfThreads, smem, s>>>(a, w, k);
        else wf_tail<false, BATCH, COND, WIDTH><<<gt, kWfThreads, smem, s>>>(a, w, k);
        hook(kPhTail, false, k);
        launches += 1;
        break;
      }
      if (k <= a.L) {
        hook(kPhShade, true, k);
        wf_shade<BATCH, COND><<<g, kWfThreads, 0, s>>>(a, w, k);
        hook(kPhShade, false, k);
        launches += 1;
      }
    }
  } else if (!BATCH) {
    for (int k = 1; k <= a.L; ++k) {
      hook(kPhTrace, true, k);
      if (stats) wf_trace<true><<<g, kWfThreads, smem, s>>>(a, w, k);
      else wf_trace<false><<<g, kWfThreads, smem, s>>>(a, w, k);
      hook(kPhTrace, false, k);
      hook(kPhShade, true, k);
      wf_shade<false, COND><<<g, kWfThreads, 0, s>>>(a, w, k);
      hook(kPhShade, false, k);
      hook(kPhShadow, true, k);
      if (stats) wf_shadow<true><<<g, kWfThreads, smem, s>>>(a, w, k);
      else wf_shadow<false><<<g, kWfThreads, smem, s>>>(a, w, k);
      hook(kPhShadow, false, k);
      launches += 3;
    }
  }
  hook(kPhFinish, true);
  wf_finish<BATCH><<<g, kWfThreads, 0, s>>>(a, w, mode, p_out);
  hook(kPhFinish, false);
  hook(kPhAdjoint, true);
  wf_adjoint<BATCH, COND><<<g, kWfThreads, 0, s>>>(a, w);
  hook(kPhAdjoint, false);
  return launches + 2;
}

}  // namespace

size_t wf_bytes(unsigned long long N, int L) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return a(N * 64) + a(N * 4) + 2 * a(N * 4) + a(N * sizeof(ShadowRec)) + a((size_t)(kMaxPathLen + 1) * N * 4) +
         a(kWfCounts * 4) + a((size_t)L * 3 * N * 16);
}

WfBuffers wf_carve(void* base, unsigned long long N, int L) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = static_cast<char*>(base);
  WfBuffers w;
  w.slot = reinterpret_cast<float4*>(p); p += a(N * 64);
  w.hit = reinterpret_cast<int*>(p); p += a(N * 4);
  w.queue[0] = reinterpret_cast<uint32_t*>(p); p += a(N * 4);
  w.queue[1] = reinterpret_cast<uint32_t*>(p); p += a(N * 4);
  w.shadow = reinterpret_cast<ShadowRec*>(p); p += a(N * sizeof(ShadowRec));
  w.adj = reinterpret_cast<uint32_t*>(p); p += a((size_t)(kMaxPathLen + 1) * N * 4);
  w.counts = reinterpret_cast<uint32_t*>(p); p += a(kWfCounts * 4);
  w.tape = reinterpret_cast<float4*>(p);
  return w;
}

int launch_wavefront_step(const StepArgs& a, const WfBuffers& w, bool stats, int n_sm, const WfTuning& tune,
                          const PhaseHook& hook, cudaStream_t s, WfMode mode, float* p_out, const RayOrder& order) {
  if (a.N == 0) return 0;
  StepArgs b = a;
  b.ray_keys = order.keys;
  // kernels with the conductor branches run only for scenes that have
  // conductors (the branches cost registers and code in every kernel);
  // the persistent passes walk the two-level or the 8-wide BVH where the
  // scene selects it
  if (a.two_level && !a.scenes) {
    if (a.conductors) return launch_wf<false, true, kWalkTwoLevel>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
    return launch_wf<false, false, kWalkTwoLevel>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
  }
  if (a.bvh8) {
    if (a.conductors)
      return a.scenes ? launch_wf<true, true, 8>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order)
                      : launch_wf<false, true, 8>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
    return a.scenes ? launch_wf<true, false, 8>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order)
                    : launch_wf<false, false, 8>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
  }
  if (a.conductors)
    return a.scenes ? launch_wf<true, true, 4>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order)
                    : launch_wf<false, true, 4>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
  return a.scenes ? launch_wf<true, false, 4>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order)
                  : launch_wf<false, false, 4>(b, w, stats, n_sm, tune, hook, s, mode, p_out, order);
}

}  // namespace dr
