// The bias term of the modified killing rate, L* p / p (Sec. 5.2, Eq. bias
// and Eq. adjoint-bias; the diagnostic of App. C), for an analytic target on
// T^2.
//
// L f = h (K f - f) is the generator of the continuous-time embedding of the
// local dynamics (holding rate h = 1 / dt, Eq. diffusion-restore-holding-
// rate; K the Euler-Maruyama kernel of Alg. 4: mean x + (stddev^2 / 2) s(x) +
// gamma_tilde (s_2, -s_1), covariance stddev^2 I, wrapped on the torus,
// s = grad log p).  Its adjoint applied to p is
//   (L* p)(y) = h ((K* p)(y) - p(y)),  (K* p)(y) = int p(x) K(x, y) dx,
// and with the modified killing rate the Restore estimate is biased by
// -(L* p / p) (Eq. bias).  One block per query point y sums the trapezoid
// rule over the square of half-width radius * stddev around y in FP64 (the
// term is h = 1 / dt times a ratio near 1, so single precision would drown
// it), then reduces in a fixed order.
#include "dr_internal.h"

namespace dr {

namespace {

constexpr int kBiasThreads = 256;

// g(x) and grad g(x) of the isotropic mixture on T^2 in FP64 (differences
// to the nearest image; K = 0: the constant).
DR_D double mixture2_eval(const DevMixture& M, double x0, double x1, double* g0, double* g1) {
  *g0 = 0.0;
  *g1 = 0.0;
  if (M.K == 0) return (double)M.cval;
  double g = 0.0;
  for (int k = 0; k < M.K; ++k) {
    const double s = (double)__ldg(M.sig + k), s2 = s * s;
    double e0 = x0 - (double)__ldg(M.mu + 2 * k), e1 = x1 - (double)__ldg(M.mu + 2 * k + 1);
    e0 -= rint(e0);
    e1 -= rint(e1);
    const double c = (double)__ldg(M.w + k) * exp(-0.5 * (e0 * e0 + e1 * e1) / s2) / (2.0 * kPiD * s2);
    g += c;
    *g0 -= c * e0 / s2;
    *g1 -= c * e1 / s2;
  }
  return g;
}

__global__ void __launch_bounds__(kBiasThreads) lstar_kernel(LstarArgs a) {
  const long long m = blockIdx.x;
  if (m >= a.n_pts) return;
  const double y0 = (double)a.y[2 * m], y1 = (double)a.y[2 * m + 1];
  const double half = a.radius * a.stddev, dx = 2.0 * half / (double)(a.n - 1);
  const double inv2s2 = 0.5 / (a.stddev * a.stddev);
  const double norm = 1.0 / (2.0 * kPiD * a.stddev * a.stddev);
  const double c2 = 0.5 * a.stddev * a.stddev;
  const long long nodes = (long long)a.n * a.n;
  double acc = 0.0;
  for (long long q = threadIdx.x; q < nodes; q += kBiasThreads) {
    const int i = (int)(q / a.n), jn = (int)(q % a.n);
    const double wi = (i == 0 || i == a.n - 1) ? 0.5 : 1.0;
    const double wj = (jn == 0 || jn == a.n - 1) ? 0.5 : 1.0;
    const double x0 = y0 - half + i * dx, x1 = y1 - half + jn * dx;
    double g0, g1;
    const double p = mixture2_eval(a.M, x0, x1, &g0, &g1) + a.eps;
    const double s0 = g0 / p, s1 = g1 / p;
    double e0 = y0 - (x0 + c2 * s0 + a.gamma_tilde * s1);
    double e1 = y1 - (x1 + c2 * s1 - a.gamma_tilde * s0);
    e0 -= rint(e0);
    e1 -= rint(e1);
    acc += wi * wj * p * norm * exp(-(e0 * e0 + e1 * e1) * inv2s2);
  }
  // fixed-order reduction: warp trees, then the warps in order
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double part[kBiasThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int w = 0; w < kBiasThreads / 32; ++w) total += part[w];
    double g0, g1;
    const double py = mixture2_eval(a.M, y0, y1, &g0, &g1) + a.eps;
    a.out[m] = a.h * (total * dx * dx / py - 1.0);
  }
}

}  // namespace

void launch_lstar(const LstarArgs& a, cudaStream_t s) {
  if (a.n_pts <= 0) return;
  lstar_kernel<<<(unsigned)a.n_pts, kBiasThreads, 0, s>>>(a);
}

}  // namespace dr
