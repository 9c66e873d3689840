// Restore chain kernels: one thread per chain, structure-of-arrays state.
//
// step_kernel fuses, per chain and step (Alg. 2 with Alg. 4 and the
// Accumulate procedure of Alg. 1):
//   a1 load state / Philox draws,
//   a2 regeneration from mu = U(T^d) if the chain was killed,
//   a3 LocalDynamics: x += (stddev^2/2) s + gamma_tilde (s_2, -s_1)
//      + stddev xi per coordinate pair, then the torus wrap,
//   a4 the path contribution f(x), p = lum(f) + eps and the pixel,
//   a6 the hold/kill clock with h = 1 / dt and k = k0 / p
//      (Eq. modified-killing-rate with uniform mu), or its Rao-Blackwellised
//      form (weight 1 / (h + k), killed with probability k / (h + k)),
//   a7 the splat record dt * f / p,
//   a5 (adjoint drift) grad log p at the new x for the next step, computed
//      only for chains that survived.
// Kill counts and ray counts are reduced per block (warp shuffles, then one
// integer atomic per block); no per-lane global atomics.
#include "dr_step.cuh"

namespace dr {

namespace {

constexpr int kStepThreads = 128;
constexpr int kStack = kTraversalStack;

struct XPerturbed {
  const float* x;
  unsigned long long N, j;
  int k;
  float v;
  DR_D float operator()(int i) const { return i == k ? v : x[(size_t)i * N + j]; }
};

struct XRow {
  const float* x;
  int d;
  long long j;
  DR_D float operator()(int i) const { return x[(size_t)j * d + i]; }
};

struct GRow {
  float* g;
  int d;
  long long j;
  DR_D void operator()(int i, float v) const { g[(size_t)j * d + i] = v; }
};

struct GNone {
  DR_D void operator()(int, float) const {}
};

DR_D double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Evaluates f, p and (optionally) grad log p through GW.
template <bool TAPE, bool STATS, bool COND = true, class XA, class GW>
DR_D float3 evaluate(const DevScene& S, const DevMixture& M, int target, int L, float eps, const XA& xa, int* pix,
                     float* p_out, bool want_grad, const GW& gw, TraceStack<kStack> st, uint32_t* err,
                     TraceStats* stats, uint32_t* rays) {
  if (target == 1) {
    const float g = mixture_eval(M, xa, eps, want_grad, gw);
    *pix = pixel_of(xa(0), xa(1), M.W, M.H);
    *p_out = g + eps;
    return f3(g, g, g);
  }
  Tape<kMaxPathLen> tape;
  const PathResult r = path_forward<kStack, STATS, TAPE, COND>(S, xa, L, &tape, st, err, stats);
  *rays += r.rays;
  *pix = r.pix;
  const float p = lum(r.f) + eps;
  *p_out = p;
  if (TAPE && want_grad) path_adjoint<COND>(S, xa, L, p, LocalTape<kMaxPathLen>{&tape}, r.nseg, gw);
  return r.f;
}

// MALA proposal of chain j (the comparison method of Sec. 6): y = x +
// (stddev^2 / 2) s(x) + stddev xi, wrapped, into the proposal array; the
// normals are Alg. 4's (same Philox blocks and pairs), without the rotation.
DR_D void mala_propose(const StepArgs& a, const Rng& rng, uint32_t step, unsigned long long j, uint32_t cj, int d) {
  const float c2 = 0.5f * a.stddev * a.stddev;
  const size_t N = a.N;
  for (int blk = 0; 4 * blk < d; ++blk) {
    const U4 r = rng.draw(step, cj, (uint32_t)blk, kNormal);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c0 = 4 * blk + 2 * h;
      if (c0 + 1 >= d) break;
      const float2 xi = box_muller(u01(h ? r.c : r.a), u01(h ? r.d : r.b));
      const size_t i0 = (size_t)c0 * N + j, i1 = i0 + N;
      a.xp[i0] = wrap01(a.x[i0] + c2 * a.score[i0] + a.stddev * xi.x);
      a.xp[i1] = wrap01(a.x[i1] + c2 * a.score[i1] + a.stddev * xi.y);
    }
  }
}

// log of the Metropolis-Hastings ratio of the MALA move x -> y in FP64:
// log p(y) - log p(x) + (|y - x - c s(x)|^2 - |x - y - c s(y)|^2) / (2 stddev^2),
// c = stddev^2 / 2, torus differences to the nearest image.
DR_D double mala_log_ratio(const StepArgs& a, unsigned long long j, int d, double px, double py) {
  const double c2 = 0.5 * (double)a.stddev * (double)a.stddev;
  double fwd = 0.0, rev = 0.0;
  for (int i = 0; i < d; ++i) {
    const size_t k = (size_t)i * a.N + j;
    const double xv = a.x[k], yv = a.xp[k];
    double e1 = yv - xv;
    e1 -= rint(e1);
    e1 -= c2 * (double)a.score[k];
    double e2 = xv - yv;
    e2 -= rint(e2);
    e2 -= c2 * (double)a.sp[k];
    fwd += e1 * e1;
    rev += e2 * e2;
  }
  const double s2 = (double)a.stddev * (double)a.stddev;
  return log(py) - log(px) + (fwd - rev) / (2.0 * s2);
}

template <int DRIFT, bool STATS, bool COND>
__global__ void __launch_bounds__(kStepThreads) step_kernel(StepArgs a) {
  extern __shared__ int smem[];
  TraceStack<kStack> st{smem + threadIdx.x, (int)blockDim.x};
  // thread t works on chain order[t] (or t); all state is indexed by chain
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < a.N;
  const unsigned long long j = active && a.order ? (unsigned long long)a.order[t].y : t;
  uint32_t err = 0, rays = 0;
  TraceStats stats{0u, 0u};
  unsigned long long kill = 0;
  double pval = 0.0;
  if (active) {
    const uint32_t cj = (uint32_t)j;
    const uint32_t step = step_index(a);
    const bool regen = a.init || a.killed[j];
    const bool mala_move = DRIFT == kDriftMala && !regen && !a.estimate_only;
    if (mala_move) mala_propose(a, rng_of(a), step, j, cj, a.d);
    else evolve_x(a, rng_of(a), step, j, cj, a.d, regen);
    const XSoA xa{a.x, a.N, j};
    int pix;
    float p;
    float3 f;
    const U4 rc = rng_of(a).draw(step, cj, 0u, kClock);
    const float u1 = u01(rc.a), u2 = u01(rc.b);
    bool killed = false;
    float wt = 0.0f;
    if (DRIFT == kDriftMala && !a.estimate_only) {
      if (mala_move) {
        // evaluate the proposal and its score, then accept or keep x
        int pix_y;
        float p_y;
        const XSoA ya{a.xp, a.N, j};
        const float3 f_y = evaluate<true, STATS, COND>(a.S, a.M, a.target, a.L, a.eps, ya, &pix_y, &p_y, true,
                                                        GSoA{a.sp, a.N, j}, st, &err, &stats, &rays);
        const float4 c = a.cur[j];
        const float p_x = lum(f3(c.x, c.y, c.z)) + a.eps;
        const double log_alpha = mala_log_ratio(a, j, a.d, (double)p_x, (double)p_y);
        const U4 rm = rng_of(a).draw(step, cj, 0u, kMH);
        if ((double)u01(rm.a) < exp(log_alpha)) {
          for (int i = 0; i < a.d; ++i) {
            const size_t k = (size_t)i * a.N + j;
            a.x[k] = a.xp[k];
            a.score[k] = a.sp[k];
          }
          f = f_y;
          p = p_y;
          pix = pix_y;
          a.cur[j] = make_float4(f.x, f.y, f.z, __int_as_float(pix));
        } else {
          f = f3(c.x, c.y, c.z);
          p = p_x;
          pix = __float_as_int(c.w);
        }
        kill_clock(a.rb, u1, u2, p, a.h, k0_of(a), &killed, &wt);
      } else if (a.target == 0) {
        // a regenerated chain: its state and, if it survives, its score
        // (forward with tape, clock, adjoint for survivors)
        Tape<kMaxPathLen> tape;
        const PathResult r = path_forward<kStack, STATS, true, COND>(a.S, xa, a.L, &tape, st, &err, &stats);
        rays += r.rays;
        pix = r.pix;
        f = r.f;
        p = lum(f) + a.eps;
        kill_clock(a.rb, u1, u2, p, a.h, k0_of(a), &killed, &wt);
        a.cur[j] = make_float4(f.x, f.y, f.z, __int_as_float(pix));
        if (!killed) path_adjoint<COND>(a.S, xa, a.L, p, LocalTape<kMaxPathLen>{&tape}, r.nseg, GSoA{a.score, a.N, j});
      } else {
        f = evaluate<false, STATS, COND>(a.S, a.M, a.target, a.L, a.eps, xa, &pix, &p, false, GNone{}, st, &err,
                                         &stats, &rays);
        kill_clock(a.rb, u1, u2, p, a.h, k0_of(a), &killed, &wt);
        a.cur[j] = make_float4(f.x, f.y, f.z, __int_as_float(pix));
        if (!killed) mixture_eval(a.M, xa, a.eps, true, GSoA{a.score, a.N, j});
      }
    } else if (DRIFT == kDriftAdjoint && !a.estimate_only && a.target == 0) {
      // forward with tape; kill decision; adjoint only if the chain survives
      Tape<kMaxPathLen> tape;
      const PathResult r = path_forward<kStack, STATS, true, COND>(a.S, xa, a.L, &tape, st, &err, &stats);
      rays += r.rays;
      pix = r.pix;
      f = r.f;
      if (a.plen) a.plen[j] = (uint8_t)r.nseg;
      p = lum(f) + a.eps;
      kill_clock(a.rb, u1, u2, p, a.h, k0_of(a), &killed, &wt);
      if (!killed) path_adjoint<COND>(a.S, xa, a.L, p, LocalTape<kMaxPathLen>{&tape}, r.nseg, GSoA{a.score, a.N, j});
    } else {
      f = evaluate<false, STATS, COND>(a.S, a.M, a.target, a.L, a.eps, xa, &pix, &p, false, GNone{}, st, &err,
                                       &stats, &rays);
      if (!a.estimate_only) kill_clock(a.rb, u1, u2, p, a.h, k0_of(a), &killed, &wt);
    }
    if (a.estimate_only) {
      pval = (double)p;
    } else {
      if (DRIFT == kDriftAdjoint && a.target == 1 && !killed) {
        mixture_eval(a.M, xa, a.eps, true, GSoA{a.score, a.N, j});
      }
      a.killed[j] = killed ? 1 : 0;
      a.logp[j] = logf(p);
      kill = killed ? 1ull : 0ull;
      if (a.init) pval = (double)p;
      if (a.rec) {
        const float s = wt / p;
        SplatRec rr;
        rr.pix = (uint32_t)pix;
        rr.r = f.x * s;
        rr.g = f.y * s;
        rr.b = f.z * s;
        a.rec[j] = rr;
      }
      if (!(isfinite(p) && isfinite(f.x) && isfinite(f.y) && isfinite(f.z))) err |= kErrNonFinite;
    }
  }
  // counters: warp sums, then one integer atomic per warp (no block barrier,
  // so warps that finish early do not wait for the block's slowest warp)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long wk = warp_sum_u64(kill), wr = warp_sum_u64(rays);
  if (err) atomicOr(a.err, err);
  if (lane == 0) {
    if (wk && a.tour_count) atomicAdd(a.tour_count, wk);
    if (wr && a.rays) atomicAdd(a.rays, wr);
  }
  if (STATS) {
    const unsigned long long wn = warp_sum_u64(stats.nodes), wt = warp_sum_u64(stats.tris);
    if (lane == 0 && a.node_visits) atomicAdd(a.node_visits, wn);
    if (lane == 0 && a.tri_tests) atomicAdd(a.tri_tests, wt);
  }
  if (a.p_partial) {
    // init only: FP64 sum of p in a fixed order (deterministic p_lambda)
    __shared__ double sp[kStepThreads / 32];
    const double wp = warp_sum_f64(pval);
    if (lane == 0) sp[warp] = wp;
    __syncthreads();
    if (threadIdx.x == 0) {
      double P = 0.0;
      for (int w = 0; w < kStepThreads / 32; ++w) P += sp[w];
      a.p_partial[blockIdx.x] = P;
    }
  }
}

// Work order for the next step: key = (killed last step, previous path
// length), so that warps get chains of similar cost; pairs (key, chain).
__global__ void order_keys_kernel(const uint8_t* __restrict__ killed, const uint8_t* __restrict__ plen,
                                  unsigned long long N, uint2* __restrict__ keys) {
  const unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const uint32_t k = ((uint32_t)killed[j] << 5) | min((uint32_t)plen[j], 31u);
  keys[j] = make_uint2(k, (uint32_t)j);
}

// Central finite differences of log p for every (coordinate, surviving
// chain): thread t -> coordinate t / N, chain t % N.
__global__ void __launch_bounds__(kStepThreads) fd_kernel(FdArgs a) {
  extern __shared__ int smem[];
  TraceStack<kStack> st{smem + threadIdx.x, (int)blockDim.x};
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long total = a.N * (unsigned long long)a.d;
  uint32_t err = 0, rays = 0;
  if (t < total) {
    const unsigned long long j = t % a.N;
    const int i = (int)(t / a.N);
    if (!a.killed[j]) {
      const float xi = a.x[(size_t)i * a.N + j];
      TraceStats stats{0u, 0u};
      int pix;
      float pp, pm;
      evaluate<false, false>(a.S, a.M, a.target, a.L, a.eps, XPerturbed{a.x, a.N, j, i, wrap01(xi + a.fd_h)}, &pix,
                             &pp, false, GNone{}, st, &err, &stats, &rays);
      evaluate<false, false>(a.S, a.M, a.target, a.L, a.eps, XPerturbed{a.x, a.N, j, i, wrap01(xi - a.fd_h)}, &pix,
                             &pm, false, GNone{}, st, &err, &stats, &rays);
      a.score[(size_t)i * a.N + j] = (logf(pp) - logf(pm)) / (2.0f * a.fd_h);
    }
  }
  const unsigned long long wr = warp_sum_u64(rays);
  if ((threadIdx.x & 31) == 0 && wr && a.rays) atomicAdd(a.rays, wr);
  if (err) atomicOr(a.err, err);
}

__global__ void __launch_bounds__(kStepThreads) eval_kernel(EvalArgs a) {
  extern __shared__ int smem[];
  TraceStack<kStack> st{smem + threadIdx.x, (int)blockDim.x};
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.Mpts) return;
  uint32_t err = 0, rays = 0;
  TraceStats stats{0u, 0u};
  int pix;
  float p;
  const XRow xa{a.x, a.d, j};
  float3 f;
  if (a.grad) f = evaluate<true, false>(a.S, a.M, a.target, a.L, a.eps, xa, &pix, &p, true, GRow{a.grad, a.d, j}, st,
                                        &err, &stats, &rays);
  else f = evaluate<false, false>(a.S, a.M, a.target, a.L, a.eps, xa, &pix, &p, false, GNone{}, st, &err, &stats,
                                  &rays);
  a.logp[j] = logf(p);
  if (a.pix) a.pix[j] = pix;
  if (a.f) { a.f[3 * j] = f.x; a.f[3 * j + 1] = f.y; a.f[3 * j + 2] = f.z; }
  if (err) atomicOr(a.err, err);
}

template <int STACK>
__global__ void __launch_bounds__(kStepThreads) trace_kernel(DevScene S, const float* __restrict__ rays, long long n,
                                                             int exclude, int* __restrict__ tri, float* __restrict__ t,
                                                             uint32_t* errp) {
  extern __shared__ int smem[];
  TraceStack<STACK> st{smem + threadIdx.x, (int)blockDim.x};
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* r = rays + 6 * i;
  uint32_t err = 0;
  float th;
  const Ray ray = make_ray(f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]));
  // the two-level or 8-wide BVH where the scene selects it (the persistent
  // passes' walk)
  const int h = S.tl_nodes ? trace_closest<STACK, false, kWalkTwoLevel>(S, ray, exclude, &th, st, &err, nullptr)
                : S.nodes8 ? trace_closest<STACK, false, 8>(S, ray, exclude, &th, st, &err, nullptr)
                           : trace_closest<STACK, false>(S, ray, exclude, &th, st, &err, nullptr);
  tri[i] = h;
  t[i] = h >= 0 ? th : __int_as_float(0x7f800000);
  if (err) atomicOr(errp, err);
}

// The same queries with each ray's walk counted: node steps (inner nodes
// visited) and triangle tests, the quantities the statistics pass sums.
template <int STACK>
__global__ void __launch_bounds__(kStepThreads) trace_stats_kernel(DevScene S, const float* __restrict__ rays,
                                                                   long long n, int exclude, int* __restrict__ tri,
                                                                   float* __restrict__ t, uint32_t* __restrict__ nodes,
                                                                   uint32_t* __restrict__ tests, uint32_t* errp) {
  extern __shared__ int smem[];
  TraceStack<STACK> st{smem + threadIdx.x, (int)blockDim.x};
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* r = rays + 6 * i;
  uint32_t err = 0;
  float th;
  TraceStats stats{0u, 0u};
  const Ray ray = make_ray(f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]));
  const int h = S.tl_nodes ? trace_closest<STACK, true, kWalkTwoLevel>(S, ray, exclude, &th, st, &err, &stats)
                : S.nodes8 ? trace_closest<STACK, true, 8>(S, ray, exclude, &th, st, &err, &stats)
                           : trace_closest<STACK, true>(S, ray, exclude, &th, st, &err, &stats);
  tri[i] = h;
  t[i] = h >= 0 ? th : __int_as_float(0x7f800000);
  nodes[i] = stats.nodes;
  tests[i] = stats.tris;
  if (err) atomicOr(errp, err);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i], key[2 * i + 1]);
  out[4 * i] = r.a;
  out[4 * i + 1] = r.b;
  out[4 * i + 2] = r.c;
  out[4 * i + 3] = r.d;
}

// Ordinary Monte Carlo over the same f (the paper's PT method, Sec. 6):
// thread t handles pixel t % n_pix and samples [c * spc, (c + 1) * spc) of
// chunk c = t / n_pix; film pair stratified to the pixel, other coordinates
// uniform from Philox (counter = (sample, pixel, block, frame<<4 | 3)).
// part[c][pix][3] receives the chunk's FP64 sum of f / (W H).
__global__ void __launch_bounds__(kStepThreads) pt_kernel(DevScene S, int L, int d, uint32_t spp, uint32_t spc,
                                                          int n_chunks, Rng rng, double* __restrict__ part,
                                                          unsigned long long* rays_out, uint32_t* errp) {
  extern __shared__ int smem[];
  TraceStack<kStack> st{smem + threadIdx.x, (int)blockDim.x};
  const long long n_pix = (long long)S.W * S.H;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t err = 0, rays = 0;
  if (t < n_pix * n_chunks) {
    const int pix = (int)(t % n_pix), c = (int)(t / n_pix);
    const int row = pix / S.W, col = pix % S.W;
    const uint32_t s0 = (uint32_t)c * spc, s1 = min(spp, s0 + spc);
    const double inv_wh = 1.0 / (double)n_pix;
    double acc[3] = {0.0, 0.0, 0.0};
    float xs[kMaxDim];
    for (uint32_t s = s0; s < s1; ++s) {
      for (int i = 0; i < d; i += 4) {
        const U4 r = rng.draw(s, (uint32_t)pix, (uint32_t)(i >> 2), kPT);
        const uint32_t w[4] = {r.a, r.b, r.c, r.d};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i + k < d) xs[i + k] = u01(w[k]);
      }
      xs[0] = ((float)col + xs[0]) / (float)S.W;
      xs[1] = ((float)row + xs[1]) / (float)S.H;
      TraceStats stats{0u, 0u};
      Tape<kMaxPathLen> tape;
      const PathResult pr =
          path_forward<kStack, false, false>(S, [&](int i) { return xs[i]; }, L, &tape, st, &err, &stats);
      rays += pr.rays;
      acc[0] += (double)pr.f.x * inv_wh;
      acc[1] += (double)pr.f.y * inv_wh;
      acc[2] += (double)pr.f.z * inv_wh;
    }
    double* o = part + ((size_t)c * n_pix + pix) * 3;
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
  }
  const unsigned long long wr = warp_sum_u64(rays);
  if ((threadIdx.x & 31) == 0 && wr && rays_out) atomicAdd(rays_out, wr);
  if (err) atomicOr(errp, err);
}

// mean[pix][c] = sum over chunks of part[chunk][pix][c] / spp (fixed order)
__global__ void pt_reduce_kernel(const double* __restrict__ part, long long n, int n_chunks, double inv_spp,
                                 double* __restrict__ mean) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < n_chunks; ++c) s += part[(size_t)c * n + i];
  mean[i] = s * inv_spp;
}

__global__ void sum_doubles_kernel(const double* __restrict__ in, int n, double* __restrict__ out) {
  // one thread, fixed order: deterministic
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += in[i];
  *out = s;
}

template <int DRIFT, bool STATS>
void launch_step_t(const StepArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)((a.N + kStepThreads - 1) / kStepThreads);
  // the conductor branches are compiled in only where a scene needs them
  if (a.conductors) step_kernel<DRIFT, STATS, true><<<grid, kStepThreads, step_smem_bytes(), s>>>(a);
  else step_kernel<DRIFT, STATS, false><<<grid, kStepThreads, step_smem_bytes(), s>>>(a);
}

}  // namespace

int step_block_size() { return kStepThreads; }
size_t step_smem_bytes() { return (size_t)kStack * kStepThreads * sizeof(int); }

__global__ void advance_step_kernel(uint32_t* step) { *step += 1u; }

void launch_advance_step(uint32_t* step, cudaStream_t s) { advance_step_kernel<<<1, 1, 0, s>>>(step); }

void launch_order_keys(const uint8_t* killed, const uint8_t* plen, unsigned long long N, uint2* keys,
                       cudaStream_t s) {
  if (N == 0) return;
  order_keys_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(killed, plen, N, keys);
}

void launch_step(const StepArgs& a, bool stats, cudaStream_t s) {
  if (a.N == 0) return;
  if (a.drift == kDriftMala) {
    if (stats) launch_step_t<kDriftMala, true>(a, s); else launch_step_t<kDriftMala, false>(a, s);
  } else if (a.drift == kDriftAdjoint) {
    if (stats) launch_step_t<kDriftAdjoint, true>(a, s); else launch_step_t<kDriftAdjoint, false>(a, s);
  } else {
    if (stats) launch_step_t<kDriftNone, true>(a, s); else launch_step_t<kDriftNone, false>(a, s);
  }
}

void launch_fd_score(const FdArgs& a, cudaStream_t s) {
  const unsigned long long total = a.N * (unsigned long long)a.d;
  if (total == 0) return;
  fd_kernel<<<(unsigned)((total + kStepThreads - 1) / kStepThreads), kStepThreads, step_smem_bytes(), s>>>(a);
}

void launch_eval(const EvalArgs& a, cudaStream_t s) {
  if (a.Mpts <= 0) return;
  eval_kernel<<<(unsigned)((a.Mpts + kStepThreads - 1) / kStepThreads), kStepThreads, step_smem_bytes(), s>>>(a);
}

void launch_trace(const DevScene& S, const float* rays, long long n, int exclude, int* tri, float* t, uint32_t* err,
                  cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = (unsigned)((n + kStepThreads - 1) / kStepThreads);
  if (S.tl_nodes)
    trace_kernel<kTraversalStackTL><<<g, kStepThreads, (size_t)kTraversalStackTL * kStepThreads * sizeof(int), s>>>(
        S, rays, n, exclude, tri, t, err);
  else
    trace_kernel<kStack><<<g, kStepThreads, step_smem_bytes(), s>>>(S, rays, n, exclude, tri, t, err);
}

void launch_trace_stats(const DevScene& S, const float* rays, long long n, int exclude, int* tri, float* t,
                        uint32_t* nodes, uint32_t* tests, uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = (unsigned)((n + kStepThreads - 1) / kStepThreads);
  if (S.tl_nodes)
    trace_stats_kernel<kTraversalStackTL>
        <<<g, kStepThreads, (size_t)kTraversalStackTL * kStepThreads * sizeof(int), s>>>(S, rays, n, exclude, tri, t,
                                                                                         nodes, tests, err);
  else
    trace_stats_kernel<kStack><<<g, kStepThreads, step_smem_bytes(), s>>>(S, rays, n, exclude, tri, t, nodes, tests,
                                                                           err);
}

void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, long long n, cudaStream_t s) {
  if (n <= 0) return;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, key, out, n);
}

void launch_pt(const DevScene& S, int L, uint32_t spp, int n_chunks, Rng rng, double* part, double* mean,
               unsigned long long* rays, uint32_t* err, cudaStream_t s) {
  const long long n_pix = (long long)S.W * S.H;
  const uint32_t spc = (spp + n_chunks - 1) / n_chunks;
  const long long threads = n_pix * n_chunks;
  const int d = 2 + 4 * (L - 1);
  pt_kernel<<<(unsigned)((threads + kStepThreads - 1) / kStepThreads), kStepThreads, step_smem_bytes(), s>>>(
      S, L, d, spp, spc, n_chunks, rng, part, rays, err);
  pt_reduce_kernel<<<(unsigned)((n_pix * 3 + 255) / 256), 256, 0, s>>>(part, n_pix * 3, n_chunks, 1.0 / spp, mean);
}

// FP64 block sums of p[0..N) over blocks of the fused kernel's size, in the
// fused kernel's order (lanes by shuffle tree, then warps in order), so a p
// estimate from stored values equals the one the fused kernel reduces.
__global__ void __launch_bounds__(kStepThreads) block_sums_kernel(const float* __restrict__ p, unsigned long long N,
                                                                  double* __restrict__ partial) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double v = t < N ? (double)p[t] : 0.0;
  __shared__ double sp[kStepThreads / 32];
  const double wp = warp_sum_f64(v);
  if ((threadIdx.x & 31) == 0) sp[threadIdx.x >> 5] = wp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double P = 0.0;
    for (int w = 0; w < kStepThreads / 32; ++w) P += sp[w];
    partial[blockIdx.x] = P;
  }
}

void launch_block_sums(const float* p, unsigned long long N, double* partial, cudaStream_t s) {
  const unsigned grid = (unsigned)((N + kStepThreads - 1) / kStepThreads);
  block_sums_kernel<<<grid, kStepThreads, 0, s>>>(p, N, partial);
}

void launch_sum_doubles(const double* in, int n, double* out, cudaStream_t s) {
  sum_doubles_kernel<<<1, 32, 0, s>>>(in, n, out);
}

}  // namespace dr
