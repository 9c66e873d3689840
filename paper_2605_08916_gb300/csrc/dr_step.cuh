// Per-chain pieces of one Restore step shared by the fused (one thread per
// chain-step) and the wavefront (one kernel per bounce) executions, so both
// perform the same floating-point operations.
#pragma once
#include "dr_internal.h"
#include "dr_path.cuh"

namespace dr {

// x[i] of chain j in the [d][N] state arrays
struct XSoA {
  const float* x;
  unsigned long long N, j;
  DR_D float operator()(int i) const { return x[(size_t)i * N + j]; }
};

// writes d log p / d x_i of chain j into the [d][N] score array
struct GSoA {
  float* g;
  unsigned long long N, j;
  DR_D void operator()(int i, float v) const { g[(size_t)i * N + j] = v; }
};

// The step index, Philox key and k0 of this launch: from device memory when
// the step is part of a replayed CUDA graph, else the launch arguments.
DR_D uint32_t step_index(const StepArgs& a) { return a.fp ? a.fp->step : a.step; }
DR_D Rng rng_of(const StepArgs& a) { return a.fp ? Rng{a.fp->seed_lo, a.fp->seed_hi, a.fp->frame} : a.rng; }
DR_D double k0_of(const StepArgs& a) { return a.fp ? a.fp->k0 : a.k0; }

// Evolve (Alg. 2): regeneration x ~ U(T^d) for a killed (or initialising)
// chain, else LocalDynamics (Alg. 4): for each coordinate pair
// x += (stddev^2 / 2) s + gamma_tilde (s_2, -s_1) + stddev xi, then wrap.
// j: the chain's index in the state arrays; cj: its Philox chain word; d:
// its PSS dimension; rng: its stream key.
DR_D void evolve_x(const StepArgs& a, const Rng& rng, uint32_t step, unsigned long long j, uint32_t cj, int d,
                   bool regen) {
  const float c2 = 0.5f * a.stddev * a.stddev;
  float* __restrict__ X = a.x;
  const float* __restrict__ Sc = a.score;
  const size_t N = a.N;
  // Philox block b covers coordinates 4b .. 4b + 3 either way: word e is
  // the uniform of coordinate 4b + e (regeneration), or words (0, 1) and
  // (2, 3) are the Box-Muller pairs of coordinate pairs 2b and 2b + 1
  // (LocalDynamics; pair q moves only if both its coordinates exist).  Both
  // run as one loop, so a warp holding a regenerating chain does not split;
  // a block's coordinates and scores are loaded before any is stored.
  for (int blk = 0; 4 * blk < d; ++blk) {
    const size_t i0 = (size_t)(4 * blk) * N + j;
    float xv[4], sv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool need = !regen && 4 * blk + (e | 1) < d;
      xv[e] = need ? X[i0 + e * N] : 0.0f;
      sv[e] = need ? Sc[i0 + e * N] : 0.0f;
    }
    const U4 r = rng.draw(step, cj, (uint32_t)blk, regen ? kRegen : kNormal);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c0 = 4 * blk + 2 * h;
      if (c0 >= d) break;
      const bool pair = c0 + 1 < d;
      const float ua = u01(h ? r.c : r.a), ub = u01(h ? r.d : r.b);
      const float2 xi = box_muller(ua, ub);
      const float s0 = sv[2 * h], s1 = sv[2 * h + 1];
      const float e0 = wrap01(xv[2 * h] + c2 * s0 + a.gamma_tilde * s1 + a.stddev * xi.x);
      const float e1 = wrap01(xv[2 * h + 1] + c2 * s1 - a.gamma_tilde * s0 + a.stddev * xi.y);
      if (regen || pair) X[i0 + (2 * h) * N] = regen ? ua : e0;
      if (pair) X[i0 + (2 * h + 1) * N] = regen ? ub : e1;
    }
  }
}

// The hold/kill clock (Accumulate of Alg. 1) with h = 1 / dt and k = k0 / p:
// the exponential race, or its Rao-Blackwellised form (weight 1 / (h + k),
// killed with probability k / (h + k)); the kill test and the RB weight are
// evaluated in FP64.
DR_D void kill_clock(int rb, float u1, float u2, float p, float h, double k0, bool* killed, float* wt) {
  if (rb) {
    *killed = (double)u2 * ((double)h * p + k0) < k0;
    *wt = (float)((double)p / ((double)h * p + k0));
  } else {
    const float t1 = -logf(1.0f - u1) / h;
    const float t2 = -logf(1.0f - u2) * p / (float)k0;
    *killed = !(t1 < t2);
    *wt = *killed ? t2 : t1;
  }
}

DR_D unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace dr
