// FP64 CPU oracle for the Diffusion Restore hot path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA library is checked against.  It shares no code, header, table or
// constant generator with the CUDA path, and nothing in the product path may
// call it.  Everything is double precision; gradients come from forward-mode
// dual numbers over the same templated code that computes the values.
//
// What is computed, and where the paper defines it (arxiv 2605.08916):
//   * Philox4x32-10 counter-based RNG (Sec. 4.3 cites Salmon et al. 2011,
//     "Parallel random numbers: as easy as 1, 2, 3"; written here from that
//     paper's definition of the round function and key schedule).
//   * The target: p = lum(f) + eps with eps = 1e-8 (Sec. 5, below Eq. for the
//     Langevin drift; Sec. 3 "Importance sampling" for p ~ luminance).
//   * f(x): the primary-sample-space path contribution.  The paper only says
//     that all methods share the same path sampling routines (Sec. 6 "Setup")
//     and that MCMC runs on the full PSS (Sec. 6 "Parameter choices"); the
//     concrete sampler below (unidirectional path tracing with next-event
//     estimation and balance-heuristic MIS, fixed maximum length, no Russian
//     roulette) is this project's reading, stated in the design notes.
//   * MALA Restore (the comparison method of Sec. 6): the same chains with a
//     Metropolis-adjusted Langevin move as local dynamics.
//   * Restore chains: Alg. 1 (Initialize + Accumulate), Alg. 2 (Evolve),
//     Alg. 3 (Resolve) and Alg. 4 (LocalDynamics) of Sec. 4.3 / 5.3, with the
//     modified killing rate k = k0 / p (Eq. modified-killing-rate, uniform
//     regeneration so u/u_lambda = 1), holding rate h = 1/dt
//     (Eq. diffusion-restore-holding-rate) and k0 = p_lambda / (m dt)
//     (Eq. killing-rate-constant).
//   * Analytic targets (isotropic Gaussian mixtures on the torus, constant
//     density, a density with a jump or a smoothed jump) used to pin the
//     Restore/Langevin logic against closed forms.
//   * The bias term L* p / p of the modified killing rate (Sec. 5.2,
//     Eq. bias and Eq. adjoint-bias; the diagnostic of App. C) for 2-D
//     targets, by quadrature of the Euler-Maruyama kernel of Alg. 4.
//   * Materials (Sec. 6 "Test scenes" names pbrt's diffuse, dielectric and
//     conductor): Lambertian, a GGX coat over Lambertian, a smooth
//     dielectric, and a rough GGX conductor whose Fresnel reflectance is
//     computed from the Fresnel equations in complex arithmetic.
// Pins (tests/test_oracle_*.py): closed-form moments, kill rates and images
// for the chain logic, the O(dt) decay of the discretisation bias and the
// torus wrap; BVH vs brute force, a white furnace and a form factor
// for f; pdf integrals, reciprocity, GGX energy and Fresnel closed forms for
// the materials; the dielectric branch by the n^2 radiance scaling inside
// glass in an emitting room and by where Snell's and the mirror law land
// rays through a slab; dual gradients vs central differences; fd_score vs a
// mixture's closed-form gradient, the dual gradient and the torus seam;
// L* p / p vs the Gaussian closed form, mass conservation and the O(dt) of
// Sec. 5.2 on a smooth density; MALA Restore exact across a jump, for a
// mixture at a large step and on the Cornell image at the paper's stddev;
// Philox vs an independent implementation.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- Philox
// Philox4x32 with 10 rounds.  Round: two 32x32->64 products of the counter's
// words 0 and 2 with the multipliers, outputs permuted and xored with the
// other counter words and the key; the key is bumped by the Weyl constants
// between rounds.
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// 24-bit uniform in [0, 1): (r >> 8) * 2^-24 (exact in float and double).
inline double u01(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

enum Purpose : uint32_t { P_REGEN = 0, P_NORMAL = 1, P_CLOCK = 2, P_PT = 3, P_MH = 4 };

struct Stream {
  uint32_t key[2];
  uint32_t frame;
  void draw(uint32_t step, uint32_t chain, uint32_t block, uint32_t purpose, uint32_t out[4]) const {
    uint32_t c[4] = {step, chain, block, (frame << 4) | purpose};
    philox4x32_10(c, key, out);
  }
};

// ---------------------------------------------------------------- duals
template <int N>
struct Dual {
  double v;
  double g[N];
  Dual() : v(0) { std::memset(g, 0, sizeof(g)); }
  Dual(double a) : v(a) { std::memset(g, 0, sizeof(g)); }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] + b.g[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] - b.g[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) { Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.g[i] = -a.g[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v / b.v; double ib = 1.0 / b.v; for (int i = 0; i < N; ++i) r.g[i] = (a.g[i] - r.v * b.g[i]) * ib; return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> inline Dual<N> operator+(double b, const Dual<N>& a) { return a + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> inline Dual<N> operator-(double b, const Dual<N>& a) { Dual<N> r = -a; r.v += b; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { Dual<N> r; r.v = a.v * b; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * b; return r; }
template <int N> inline Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) { Dual<N> r; r.v = std::sqrt(a.v); double k = r.v > 0 ? 0.5 / r.v : 0.0; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * k; return r; }
template <int N> inline Dual<N> log(const Dual<N>& a) { Dual<N> r; r.v = std::log(a.v); double k = 1.0 / a.v; for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * k; return r; }
template <int N> inline Dual<N> exp(const Dual<N>& a) { Dual<N> r; r.v = std::exp(a.v); for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * r.v; return r; }
template <int N> inline Dual<N> sin(const Dual<N>& a) { Dual<N> r; r.v = std::sin(a.v); double k = std::cos(a.v); for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * k; return r; }
template <int N> inline Dual<N> cos(const Dual<N>& a) { Dual<N> r; r.v = std::cos(a.v); double k = -std::sin(a.v); for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * k; return r; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> inline Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) { a = a * b; return a; }
template <int N> inline double val(const Dual<N>& a) { return a.v; }
inline double val(double a) { return a; }
using std::sqrt; using std::log; using std::exp; using std::sin; using std::cos;

template <class T>
struct V3 {
  T x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(T a, T b, T c) : x(a), y(b), z(c) {}
  template <class U> static V3 from(const V3<U>& o) { return V3(T(o.x), T(o.y), T(o.z)); }
};
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> inline V3<T> operator-(const V3<T>& a) { return V3<T>(-a.x, -a.y, -a.z); }
template <class T, class S> inline V3<T> operator*(const V3<T>& a, const S& s) { return V3<T>(a.x * s, a.y * s, a.z * s); }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) { return V3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
template <class T> inline V3<T> normalize(const V3<T>& a) { T l = sqrt(dot(a, a)); return V3<T>(a.x / l, a.y / l, a.z / l); }
template <class T> inline V3<double> vval(const V3<T>& a) { return V3<double>(val(a.x), val(a.y), val(a.z)); }
template <class T> inline V3<T> lift(const V3<double>& a) { return V3<T>(T(a.x), T(a.y), T(a.z)); }

using D3 = V3<double>;

// Rec. 709 luminance.
constexpr double LUM[3] = {0.2126, 0.7152, 0.0722};
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- scene
enum MatType { M_DIFFUSE = 0, M_GLOSSY = 1, M_DIELECTRIC = 2, M_EMITTER = 3, M_CONDUCTOR = 4 };
// Conductor records reuse the albedo slots for the real part eta of the
// complex index of refraction (RGB) and slots 9..11 for its imaginary part k.
struct Mat {
  int type;
  double albedo[3], rough, ior, emit[3], f0, k[3];
  bool emissive() const { return emit[0] > 0 || emit[1] > 0 || emit[2] > 0; }
};
struct Tri {
  D3 v0, v1, v2, e1, e2, N, ng, au, av;  // N = cross(e1, e2); au/av give barycentrics from P - v0
  double area;
  int mat;
  bool has_n;
  D3 n0, n1, n2;
};
struct Camera { D3 eye, fwd, right, up; double tx, ty; };

struct BvhNode { double lo[3], hi[3]; int left, right, start, count; };

struct Scene {
  std::vector<Tri> tris;
  std::vector<Mat> mats;
  Camera cam;
  int W, H;
  double tmin;
  std::vector<int> lights;        // emissive triangle ids, ascending
  std::vector<double> light_cdf;  // inclusive prefix of selection probabilities
  std::vector<double> sel;        // per triangle selection probability (0 if not a light)
  std::vector<BvhNode> nodes;
  std::vector<int> order;
  bool use_bvh;
};

// Moller-Trumbore in double.  Hit iff det != 0, u >= 0, v >= 0, u + v <= 1,
// tmin < t < tmax.
inline bool tri_hit(const Tri& tr, const D3& o, const D3& d, double tmin, double tmax, double* tout) {
  D3 p = cross(d, tr.e2);
  double det = dot(tr.e1, p);
  if (det == 0.0) return false;
  double inv = 1.0 / det;
  D3 tv = o - tr.v0;
  double u = dot(tv, p) * inv;
  if (u < 0.0 || u > 1.0) return false;
  D3 q = cross(tv, tr.e1);
  double v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  double t = dot(tr.e2, q) * inv;
  if (!(t > tmin && t < tmax)) return false;
  *tout = t;
  return true;
}

inline bool box_hit(const BvhNode& n, const D3& o, const D3& inv, double tmax) {
  double t0 = 0.0, t1 = tmax;
  const double oo[3] = {o.x, o.y, o.z}, ii[3] = {inv.x, inv.y, inv.z};
  for (int a = 0; a < 3; ++a) {
    double ta = (n.lo[a] - oo[a]) * ii[a], tb = (n.hi[a] - oo[a]) * ii[a];
    if (ta > tb) std::swap(ta, tb);
    if (std::isnan(ta)) ta = -INFINITY;
    if (std::isnan(tb)) tb = INFINITY;
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1 * (1.0 + 1e-12) + 1e-12) return false;
  }
  return true;
}

void build_bvh(Scene& S) {
  int n = (int)S.tris.size();
  S.order.resize(n);
  std::iota(S.order.begin(), S.order.end(), 0);
  std::vector<D3> cen(n);
  for (int i = 0; i < n; ++i) { const Tri& t = S.tris[i]; cen[i] = (t.v0 + t.v1 + t.v2) * (1.0 / 3.0); }
  S.nodes.clear();
  S.nodes.reserve(2 * n / 2 + 2);
  struct Item { int node, start, count; };
  std::vector<Item> stack;
  S.nodes.push_back(BvhNode{});
  stack.push_back({0, 0, n});
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    BvhNode nd{};
    for (int a = 0; a < 3; ++a) { nd.lo[a] = INFINITY; nd.hi[a] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = it.start; k < it.start + it.count; ++k) {
      const Tri& t = S.tris[S.order[k]];
      const D3* vs[3] = {&t.v0, &t.v1, &t.v2};
      for (int j = 0; j < 3; ++j) {
        const double c[3] = {vs[j]->x, vs[j]->y, vs[j]->z};
        for (int a = 0; a < 3; ++a) { nd.lo[a] = std::min(nd.lo[a], c[a]); nd.hi[a] = std::max(nd.hi[a], c[a]); }
      }
      const double cc[3] = {cen[S.order[k]].x, cen[S.order[k]].y, cen[S.order[k]].z};
      for (int a = 0; a < 3; ++a) { clo[a] = std::min(clo[a], cc[a]); chi[a] = std::max(chi[a], cc[a]); }
    }
    if (it.count <= 4) {
      nd.left = nd.right = -1;
      nd.start = it.start;
      nd.count = it.count;
      S.nodes[it.node] = nd;
      continue;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    int mid = it.start + it.count / 2;
    auto key = [&](int i) { return axis == 0 ? cen[i].x : axis == 1 ? cen[i].y : cen[i].z; };
    std::nth_element(S.order.begin() + it.start, S.order.begin() + mid, S.order.begin() + it.start + it.count,
                     [&](int a, int b) { double ka = key(a), kb = key(b); return ka < kb || (ka == kb && a < b); });
    nd.left = (int)S.nodes.size();
    nd.right = nd.left + 1;
    nd.start = nd.count = 0;
    S.nodes[it.node] = nd;
    S.nodes.push_back(BvhNode{});
    S.nodes.push_back(BvhNode{});
    stack.push_back({nd.left, it.start, mid - it.start});
    stack.push_back({nd.right, mid, it.start + it.count - mid});
  }
}

// Closest hit: smallest t; ties broken by the smallest triangle id.
inline bool finite_ray(const D3& o, const D3& d) {
  return std::isfinite(o.x) && std::isfinite(o.y) && std::isfinite(o.z) && std::isfinite(d.x) &&
         std::isfinite(d.y) && std::isfinite(d.z);
}

bool closest(const Scene& S, const D3& o, const D3& d, int exclude, int* tri, double* t, long* tests = nullptr) {
  int best = -1;
  double bt = INFINITY;
  if (!finite_ray(o, d)) return false;
  auto consider = [&](int i) {
    if (i == exclude) return;
    double th;
    if (tests) ++*tests;
    if (tri_hit(S.tris[i], o, d, S.tmin, INFINITY, &th)) {
      if (th < bt || (th == bt && i < best)) { bt = th; best = i; }
    }
  };
  if (!S.use_bvh) {
    for (int i = 0; i < (int)S.tris.size(); ++i) consider(i);
  } else {
    D3 inv(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
    std::vector<int> st;
    st.reserve(128);
    st.push_back(0);
    while (!st.empty()) {
      int ni = st.back();
      st.pop_back();
      const BvhNode& nd = S.nodes[ni];
      if (!box_hit(nd, o, inv, bt)) continue;
      if (nd.left < 0) {
        for (int k = nd.start; k < nd.start + nd.count; ++k) consider(S.order[k]);
      } else {
        st.push_back(nd.right);
        st.push_back(nd.left);
      }
    }
  }
  if (best < 0) return false;
  *tri = best;
  *t = bt;
  return true;
}

// Any hit in (tmin, tmax), ignoring two triangle ids.
bool occluded(const Scene& S, const D3& o, const D3& d, double tmax, int ex0, int ex1) {
  if (!finite_ray(o, d)) return true;
  auto test = [&](int i) {
    if (i == ex0 || i == ex1) return false;
    double th;
    return tri_hit(S.tris[i], o, d, S.tmin, tmax, &th);
  };
  if (!S.use_bvh) {
    for (int i = 0; i < (int)S.tris.size(); ++i) if (test(i)) return true;
    return false;
  }
  D3 inv(1.0 / d.x, 1.0 / d.y, 1.0 / d.z);
  std::vector<int> st;
  st.reserve(128);
  st.push_back(0);
  while (!st.empty()) {
    int ni = st.back();
    st.pop_back();
    const BvhNode& nd = S.nodes[ni];
    if (!box_hit(nd, o, inv, tmax)) continue;
    if (nd.left < 0) {
      for (int k = nd.start; k < nd.start + nd.count; ++k) if (test(S.order[k])) return true;
    } else {
      st.push_back(nd.right);
      st.push_back(nd.left);
    }
  }
  return false;
}

// ---------------------------------------------------------------- BSDFs
// Orthonormal basis around a unit normal (branchless construction of
// Duff et al. 2017, "Building an Orthonormal Basis, Revisited").
template <class T>
void onb(const V3<T>& n, V3<T>& t, V3<T>& b) {
  double s = val(n.z) >= 0.0 ? 1.0 : -1.0;
  T a = -1.0 / (s + n.z);
  T c = n.x * n.y * a;
  t = V3<T>(1.0 + s * n.x * n.x * a, s * c, -s * n.x);
  b = V3<T>(c, s + n.y * n.y * a, -n.y);
}

// GGX (Trowbridge-Reitz) normal distribution, Smith height-correlated
// masking-shadowing, Schlick Fresnel.  alpha = roughness (no remapping).
template <class T> T ggx_D(const T& nh, double alpha) {
  double a2 = alpha * alpha;
  T k = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (PI * k * k);
}
template <class T> T smith_lambda(const T& c, double alpha) {
  T c2 = c * c;
  T t2 = (1.0 - c2) / c2;
  return (sqrt(1.0 + alpha * alpha * t2) - 1.0) * 0.5;
}
constexpr double GLOSSY_SPEC_PROB = 0.5;

// Glossy ("GGX coat over Lambertian") BSDF value (RGB) and the solid-angle
// pdf of its two-lobe sampler for a pair of directions in the upper
// hemisphere of n.
template <class T>
void glossy_eval(const Mat& m, const V3<T>& n, const V3<T>& wo, const V3<T>& wi, T fs[3], T& pdf) {
  T co = dot(n, wo), ci = dot(n, wi);
  V3<T> h = normalize(wo + wi);
  T nh = dot(n, h), oh = dot(wo, h), ih = dot(wi, h);
  T D = ggx_D(nh, m.rough);
  T G = 1.0 / (1.0 + smith_lambda(co, m.rough) + smith_lambda(ci, m.rough));
  T om = 1.0 - ih;
  T om2 = om * om;
  T F = m.f0 + (1.0 - m.f0) * (om2 * om2 * om);
  T spec = D * G * F / (4.0 * co * ci);
  for (int c = 0; c < 3; ++c) fs[c] = m.albedo[c] * (1.0 - m.f0) / PI + spec;
  T oh_abs = val(oh) >= 0 ? oh : -oh;
  pdf = GLOSSY_SPEC_PROB * D * nh / (4.0 * oh_abs) + (1.0 - GLOSSY_SPEC_PROB) * ci / PI;
}

// Complex numbers over the scalar type T (values or duals), enough for the
// Fresnel equations of an absorbing interface.
template <class T>
struct Cx {
  T re, im;
  Cx(T r = T(0.0), T i = T(0.0)) : re(r), im(i) {}
};
template <class T> Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re + b.re, a.im + b.im); }
template <class T> Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re - b.re, a.im - b.im); }
template <class T> Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) {
  return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> Cx<T> operator/(const Cx<T>& a, const Cx<T>& b) {
  T q = b.re * b.re + b.im * b.im;
  return Cx<T>((a.re * b.re + a.im * b.im) / q, (a.im * b.re - a.re * b.im) / q);
}
template <class T> T norm2(const Cx<T>& a) { return a.re * a.re + a.im * a.im; }
// Principal square root.
template <class T> Cx<T> csqrt(const Cx<T>& z) {
  T r = sqrt(norm2(z));
  T re = sqrt((r + z.re) * 0.5);
  T im = sqrt((r - z.re) * 0.5);
  if (val(z.im) < 0.0) im = -im;
  return Cx<T>(re, im);
}

// Fresnel reflectance of unpolarised light arriving from vacuum at an
// interface of complex index eta + i k (a conductor), for the cosine ci of
// the angle of incidence: Snell's law with the complex index gives the
// transmitted cosine, and R = (|r_s|^2 + |r_p|^2) / 2 with the amplitude
// coefficients of the Fresnel equations.
template <class T>
T fresnel_conductor(const T& ci, double eta, double k) {
  const Cx<T> n{T(eta), T(k)};
  Cx<T> s2(1.0 - ci * ci);
  Cx<T> ct = csqrt(Cx<T>(T(1.0)) - s2 / (n * n));
  Cx<T> c(ci);
  Cx<T> rs = (c - n * ct) / (c + n * ct);
  Cx<T> rp = (n * c - ct) / (n * c + ct);
  return (norm2(rs) + norm2(rp)) * 0.5;
}

// Rough conductor (pbrt's conductor with a GGX distribution): a single
// specular microfacet lobe, D G2 F / (4 cos_o cos_i) with the conductor
// Fresnel per RGB channel, sampled by D cos(theta_h) half-vectors.
template <class T>
void conductor_eval(const Mat& m, const V3<T>& n, const V3<T>& wo, const V3<T>& wi, T fs[3], T& pdf) {
  T co = dot(n, wo), ci = dot(n, wi);
  V3<T> h = normalize(wo + wi);
  T nh = dot(n, h), oh = dot(wo, h);
  T D = ggx_D(nh, m.rough);
  T G = 1.0 / (1.0 + smith_lambda(co, m.rough) + smith_lambda(ci, m.rough));
  for (int c = 0; c < 3; ++c) fs[c] = D * G * fresnel_conductor(oh, m.albedo[c], m.k[c]) / (4.0 * co * ci);
  T oh_abs = val(oh) >= 0 ? oh : -oh;
  pdf = D * nh / (4.0 * oh_abs);
}

template <class T>
void bsdf_eval(const Mat& m, const V3<T>& n, const V3<T>& wo, const V3<T>& wi, T fs[3], T& pdf) {
  if (m.type == M_GLOSSY) { glossy_eval(m, n, wo, wi, fs, pdf); return; }
  if (m.type == M_CONDUCTOR) { conductor_eval(m, n, wo, wi, fs, pdf); return; }
  T ci = dot(n, wi);
  for (int c = 0; c < 3; ++c) fs[c] = T(m.albedo[c] / PI);
  pdf = ci / PI;
}

// Cosine-weighted hemisphere direction in the local frame (Malley's method).
template <class T>
V3<T> cosine_local(const T& u1, const T& u2) {
  T r = sqrt(u1);
  T phi = 2.0 * PI * u2;
  return V3<T>(r * cos(phi), r * sin(phi), sqrt(1.0 - u1));
}

// Samples the BSDF of an opaque material.  Returns false if the sampled
// direction is not in the upper hemisphere of both normals.
template <class T>
bool opaque_sample(const Mat& m, const V3<T>& n, const D3& ngf, const V3<T>& wo, const T& u1, const T& u2,
                   V3<T>& wi, T w[3], T& pdf, int& lobe) {
  V3<T> t, b;
  onb(n, t, b);
  if (m.type == M_GLOSSY || m.type == M_CONDUCTOR) {
    const double sp = m.type == M_CONDUCTOR ? 1.0 : GLOSSY_SPEC_PROB;
    if (val(u1) < sp) {
      lobe = 1;
      T v = u1 / sp;
      double a2 = m.rough * m.rough;
      T den = 1.0 + (a2 - 1.0) * v;
      T ch = sqrt((1.0 - v) / den);
      T sh = m.rough * sqrt(v / den);
      T phi = 2.0 * PI * u2;
      V3<T> h = t * (sh * cos(phi)) + b * (sh * sin(phi)) + n * ch;
      wi = h * (2.0 * dot(wo, h)) - wo;
    } else {
      lobe = 0;
      T v = (u1 - GLOSSY_SPEC_PROB) / (1.0 - GLOSSY_SPEC_PROB);
      V3<T> l = cosine_local(v, u2);
      wi = t * l.x + b * l.y + n * l.z;
    }
  } else {
    lobe = 0;
    V3<T> l = cosine_local(u1, u2);
    wi = t * l.x + b * l.y + n * l.z;
  }
  T ci = dot(n, wi);
  if (!(val(ci) > 0.0) || !(dot(ngf, vval(wi)) > 0.0)) return false;
  T fs[3];
  bsdf_eval(m, n, wo, wi, fs, pdf);
  for (int c = 0; c < 3; ++c) w[c] = fs[c] * ci / pdf;
  return true;
}

// Exact Fresnel reflectance of a smooth dielectric interface; eta = n_t/n_i.
double fresnel_dielectric(double ci, double ct, double eta) {
  double rs = (ci - eta * ct) / (ci + eta * ct);
  double rp = (eta * ci - ct) / (eta * ci + ct);
  return 0.5 * (rs * rs + rp * rp);
}

// ---------------------------------------------------------------- f(x)
struct PathInfo {
  static constexpr int MAXV = 20;
  int nseg = 0;
  int tri[MAXV];     // hit triangle per traced segment (-1 = miss)
  int lobe[MAXV];    // sampled lobe per vertex (0 diffuse, 1 spec, 2 reflect, 3 refract)
  int vis[MAXV];     // NEE: -1 not attempted, 0 occluded / invalid, 1 visible
  int light[MAXV];   // NEE light triangle
  int rays = 0;
};

template <class T>
struct PathOut {
  T f[3];
  int pix;
  PathInfo info;
};

// The primary-sample-space path contribution.  PSS layout (d = 2 + 4 (L - 1)):
// x[0], x[1] film position (pixel = floor(x0 W), floor(x1 H), row 0 at the
// top); for scattering vertex v = 1 .. L - 1 at base b = 2 + 4 (v - 1):
// x[b], x[b+1] BSDF sample (the first coordinate also picks the lobe, by
// rescaling), x[b+2], x[b+3] light sample (the first coordinate also picks the
// emitting triangle, by rescaling).  f carries the pixel importance W H so
// that integrating f over one pixel's film area gives the pixel's mean
// radiance.
template <class T>
void eval_path(const Scene& S, const T* x, int L, PathOut<T>& out) {
  PathInfo& info = out.info;
  for (int i = 0; i < PathInfo::MAXV; ++i) { info.tri[i] = -1; info.lobe[i] = -1; info.vis[i] = -1; info.light[i] = -1; }
  double WH = (double)S.W * (double)S.H;
  T beta[3] = {T(WH), T(WH), T(WH)};
  for (int c = 0; c < 3; ++c) out.f[c] = T(0.0);
  {
    int col = (int)std::floor(val(x[0]) * S.W), row = (int)std::floor(val(x[1]) * S.H);
    col = std::min(std::max(col, 0), S.W - 1);
    row = std::min(std::max(row, 0), S.H - 1);
    out.pix = row * S.W + col;
  }
  const Camera& C = S.cam;
  T sx = (2.0 * x[0] - 1.0) * C.tx;
  T sy = (1.0 - 2.0 * x[1]) * C.ty;
  V3<T> d = normalize(lift<T>(C.fwd) + lift<T>(C.right) * sx + lift<T>(C.up) * sy);
  V3<T> o = lift<T>(C.eye);
  int prev_tri = -1;
  bool prev_delta = true;
  T prev_pdf = T(0.0);
  for (int seg = 1; seg <= L; ++seg) {
    int tri;
    double th;
    ++info.rays;
    if (!closest(S, vval(o), vval(d), prev_tri, &tri, &th)) break;
    const Tri& tr = S.tris[tri];
    // a hit within 1e-6 (cosine) of grazing ends the path: the hit distance
    // as a function of the ray is ill-conditioned there
    if (!(std::fabs(dot(vval(d), tr.ng)) >= 1e-6)) break;
    info.nseg = seg;
    info.tri[seg - 1] = tri;
    const Mat& m = S.mats[tr.mat];
    // differentiable hit point on the (fixed) plane of the hit triangle
    V3<T> N = lift<T>(tr.N);
    T t = dot(lift<T>(tr.v0) - o, N) / dot(d, N);
    V3<T> P = o + d * t;
    if (m.emissive()) {
      T cl = -dot(lift<T>(tr.ng), d);
      if (val(cl) > 0.0) {
        T w = T(1.0);
        if (!prev_delta) {
          T pl = S.sel[tri] / tr.area * t * t / cl;
          w = prev_pdf / (prev_pdf + pl);
        }
        for (int c = 0; c < 3; ++c) out.f[c] += beta[c] * m.emit[c] * w;
      }
    }
    if (m.type == M_EMITTER || seg == L) break;
    V3<T> wo = -d;
    V3<T> ns;
    if (tr.has_n) {
      V3<T> q = P - lift<T>(tr.v0);
      T bu = dot(q, lift<T>(tr.au)), bv = dot(q, lift<T>(tr.av));
      ns = normalize(lift<T>(tr.n0) * (1.0 - bu - bv) + lift<T>(tr.n1) * bu + lift<T>(tr.n2) * bv);
    } else {
      ns = lift<T>(tr.ng);
    }
    const int b = 2 + 4 * (seg - 1);
    if (m.type == M_DIELECTRIC) {
      bool entering = dot(tr.ng, vval(wo)) > 0.0;
      V3<T> nn = entering ? ns : -ns;
      T c = dot(nn, wo);
      if (!(val(c) > 0.0)) break;
      double eta = entering ? m.ior : 1.0 / m.ior;
      T s2 = (1.0 - c * c) / (eta * eta);
      double F = 1.0;
      T ct = T(0.0);
      if (val(s2) < 1.0) {
        ct = sqrt(1.0 - s2);
        F = fresnel_dielectric(val(c), val(ct), eta);
      }
      V3<T> wi;
      double wgt;
      if (val(x[b]) < F) {
        wi = nn * (2.0 * c) - wo;
        wgt = 1.0;
        info.lobe[seg] = 2;
      } else {
        wi = wo * (-1.0 / eta) + nn * (c / eta - ct);
        wgt = 1.0 / (eta * eta);
        info.lobe[seg] = 3;
      }
      for (int k = 0; k < 3; ++k) beta[k] = beta[k] * wgt;
      prev_delta = true;
      prev_pdf = T(0.0);
      o = P;
      d = wi;
      prev_tri = tri;
      continue;
    }
    D3 ngf = tr.ng;
    if (dot(ngf, vval(wo)) < 0.0) { ngf = -ngf; ns = -ns; }
    if (!(val(dot(ns, wo)) > 0.0)) break;
    // next-event estimation: one point on one emitting triangle
    if (!S.lights.empty()) {
      T ul = x[b + 2];
      int k = 0;
      while (k + 1 < (int)S.lights.size() && !(val(ul) < S.light_cdf[k])) ++k;
      double lo = k == 0 ? 0.0 : S.light_cdf[k - 1];
      double pk = S.light_cdf[k] - lo;
      T v1 = (ul - lo) / pk;
      if (val(v1) >= 1.0) v1 = T(std::nextafter(1.0, 0.0));
      if (val(v1) < 0.0) v1 = T(0.0);
      const int lt = S.lights[k];
      const Tri& L_ = S.tris[lt];
      T su = sqrt(v1);
      T v2 = x[b + 3];
      V3<T> y = lift<T>(L_.v0) * (1.0 - su) + lift<T>(L_.v1) * (su * (1.0 - v2)) + lift<T>(L_.v2) * (su * v2);
      V3<T> wv = y - P;
      T dist2 = dot(wv, wv);
      T dist = sqrt(dist2);
      V3<T> wi = wv * (1.0 / dist);
      T ci = dot(ns, wi);
      T cl = -dot(lift<T>(L_.ng), wi);
      info.light[seg] = lt;
      info.vis[seg] = 0;
      if (val(ci) > 0.0 && val(cl) > 0.0 && dot(ngf, vval(wi)) > 0.0) {
        ++info.rays;
        if (!occluded(S, vval(P), vval(wi), val(dist) - S.tmin, tri, lt)) {
          info.vis[seg] = 1;
          T fs[3], pb;
          bsdf_eval(m, ns, wo, wi, fs, pb);
          T pl = S.sel[lt] / L_.area * dist2 / cl;
          const Mat& lm = S.mats[L_.mat];
          T g = ci / (pl + pb);
          for (int c = 0; c < 3; ++c) out.f[c] += beta[c] * fs[c] * lm.emit[c] * g;
        }
      }
    }
    // BSDF sampling
    V3<T> wi;
    T w[3], pdf;
    int lobe;
    if (!opaque_sample(m, ns, ngf, wo, x[b], x[b + 1], wi, w, pdf, lobe)) break;
    info.lobe[seg] = lobe;
    for (int c = 0; c < 3; ++c) beta[c] = beta[c] * w[c];
    prev_delta = false;
    prev_pdf = pdf;
    o = P;
    d = wi;
    prev_tri = tri;
  }
}

// ---------------------------------------------------------------- targets
struct Mixture {
  int d, K, W, H;
  std::vector<double> w, mu, sig;
  double cval;
};

// Isotropic Gaussian mixture on the torus (component differences taken to the
// nearest image); K = 0 is the constant density cval.  Returns g(x) and
// optionally its gradient.
double mixture_eval(const Mixture& M, const double* x, double* grad) {
  if (grad) std::fill(grad, grad + M.d, 0.0);
  if (M.K == 0) return M.cval;
  double g = 0.0;
  std::vector<double> del(M.d);
  for (int k = 0; k < M.K; ++k) {
    double s2 = M.sig[k] * M.sig[k], q = 0.0;
    for (int i = 0; i < M.d; ++i) {
      double dd = x[i] - M.mu[k * M.d + i];
      dd -= std::nearbyint(dd);
      del[i] = dd;
      q += dd * dd;
    }
    double c = M.w[k] * std::exp(-0.5 * q / s2) / std::pow(2.0 * PI * s2, 0.5 * M.d);
    g += c;
    if (grad) for (int i = 0; i < M.d; ++i) grad[i] -= c * del[i] / s2;
  }
  return g;
}

// A density on the torus with one jump per half period along x0 (used to
// read the bias claim of Sec. 5.2 on a discontinuous target):
// g(x) = c2 + (c1 - c2) (1 + tanh(q(x0) / w)) / 2 with q(x0) = sin(2 pi x0) / (2 pi),
// i.e. about c1 on x0 in (0, 1/2) and c2 on (1/2, 1), with transitions of
// width ~w at x0 = 0 and 1/2 (q ~ +-(x0 - edge) there).  w = 0 is the sharp
// step (the derivative of its smooth pieces is 0).  The other coordinates do
// not enter.
struct StepDensity {
  int d, W, H;
  double c1, c2, w;
};

double step_eval(const StepDensity& D, const double* x, double* grad) {
  if (grad) std::fill(grad, grad + D.d, 0.0);
  const double x0 = x[0] - std::floor(x[0]);
  if (D.w <= 0.0) {
    if (x0 == 0.0 || x0 == 0.5) return 0.5 * (D.c1 + D.c2);
    return x0 < 0.5 ? D.c1 : D.c2;
  }
  const double q = std::sin(2.0 * PI * x0) / (2.0 * PI);
  const double th = std::tanh(q / D.w);
  if (grad) grad[0] = (D.c1 - D.c2) * 0.5 * (1.0 - th * th) / D.w * std::cos(2.0 * PI * x0);
  return D.c2 + (D.c1 - D.c2) * 0.5 * (1.0 + th);
}

// ---------------------------------------------------------------- evaluation
struct Target {
  int kind;  // 0 scene, 1 mixture, 2 step density
  Scene* S;
  Mixture* M;
  int L;
  StepDensity* J = nullptr;
  int d() const { return kind == 0 ? 2 + 4 * (L - 1) : kind == 1 ? M->d : J->d; }
  int W() const { return kind == 0 ? S->W : kind == 1 ? M->W : J->W; }
  int H() const { return kind == 0 ? S->H : kind == 1 ? M->H : J->H; }
};

Target make_target(void* tgt, int kind, int L) {
  Target T{kind, kind == 0 ? static_cast<Scene*>(tgt) : nullptr, kind == 1 ? static_cast<Mixture*>(tgt) : nullptr, L};
  if (kind == 2) T.J = static_cast<StepDensity*>(tgt);
  return T;
}

struct EvalResult {
  double f[3];
  double p;
  int pix;
  PathInfo info;
};

template <int N>
void eval_grad_scene(const Scene& S, const double* x, int L, int d, double eps, EvalResult& r, double* grad) {
  std::vector<Dual<N>> xd(d);
  for (int i = 0; i < d; ++i) { xd[i] = Dual<N>(x[i]); xd[i].g[i] = 1.0; }
  PathOut<Dual<N>> po;
  eval_path(S, xd.data(), L, po);
  Dual<N> p = po.f[0] * LUM[0] + po.f[1] * LUM[1] + po.f[2] * LUM[2] + eps;
  for (int c = 0; c < 3; ++c) r.f[c] = po.f[c].v;
  r.p = p.v;
  r.pix = po.pix;
  r.info = po.info;
  for (int i = 0; i < d; ++i) grad[i] = p.g[i] / p.v;  // grad log p
}

// Evaluates f, p = lum(f) + eps, and (if grad) grad log p at x.
void evaluate(const Target& T, const double* x, double eps, EvalResult& r, double* grad) {
  const int d = T.d();
  if (T.kind == 1 || T.kind == 2) {
    std::vector<double> gg(d);
    double g = T.kind == 1 ? mixture_eval(*T.M, x, grad ? gg.data() : nullptr)
                           : step_eval(*T.J, x, grad ? gg.data() : nullptr);
    r.f[0] = r.f[1] = r.f[2] = g;
    r.p = g + eps;
    const int W = T.W(), H = T.H();
    int col = std::min(std::max((int)std::floor(x[0] * W), 0), W - 1);
    int row = std::min(std::max((int)std::floor(x[1] * H), 0), H - 1);
    r.pix = row * W + col;
    r.info = PathInfo{};
    if (grad) for (int i = 0; i < d; ++i) grad[i] = gg[i] / r.p;
    return;
  }
  if (!grad) {
    PathOut<double> po;
    eval_path(*T.S, x, T.L, po);
    for (int c = 0; c < 3; ++c) r.f[c] = po.f[c];
    r.p = LUM[0] * po.f[0] + LUM[1] * po.f[1] + LUM[2] * po.f[2] + eps;
    r.pix = po.pix;
    r.info = po.info;
    return;
  }
  if (d <= 16) eval_grad_scene<16>(*T.S, x, T.L, d, eps, r, grad);
  else if (d <= 32) eval_grad_scene<32>(*T.S, x, T.L, d, eps, r, grad);
  else if (d <= 48) eval_grad_scene<48>(*T.S, x, T.L, d, eps, r, grad);
  else eval_grad_scene<64>(*T.S, x, T.L, d, eps, r, grad);
}

// Torus wrap x - floor(x); a result that rounds to 1 becomes 0.
inline double wrap01(double v) {
  double r = v - std::floor(v);
  return r >= 1.0 ? 0.0 : r;
}

// ---------------------------------------------------------------- Restore
struct Params {
  int32_t L, drift_mode, rb_weight, pad;
  double stddev, dt, gamma_tilde, eps, fd_h, m, k0;
};
enum Drift { D_NONE = 0, D_FD = 1, D_EXACT = 2, D_MALA = 3 };

// Central finite differences of log p on the torus with step h.
void fd_score(const Target& T, const double* x, double eps, double h, double* s) {
  const int d = T.d();
  std::vector<double> xp(x, x + d);
  EvalResult ra, rb;
  for (int i = 0; i < d; ++i) {
    xp[i] = wrap01(x[i] + h);
    evaluate(T, xp.data(), eps, ra, nullptr);
    xp[i] = wrap01(x[i] - h);
    evaluate(T, xp.data(), eps, rb, nullptr);
    xp[i] = x[i];
    s[i] = (std::log(ra.p) - std::log(rb.p)) / (2.0 * h);
  }
}

struct ChainRec {
  double f[3], p, val[3];
  int pix;
  bool killed;
  PathInfo info;
};

// Accumulate (Alg. 1): f, p and pixel at x; the hold/kill race (or its
// Rao-Blackwellised form); the splat value Dt * f / p; and the score at x for
// the next LocalDynamics call when the chain survives.
void accumulate(const Target& T, const Params& P, const Stream& st, uint32_t step, uint32_t chain,
                const double* x, double* score, ChainRec& rec) {
  const int d = T.d();
  EvalResult r;
  std::vector<double> g(d, 0.0);
  const bool exact = P.drift_mode == D_EXACT || P.drift_mode == D_MALA;
  evaluate(T, x, P.eps, r, exact ? g.data() : nullptr);
  uint32_t rr[4];
  st.draw(step, chain, 0, P_CLOCK, rr);
  double u1 = u01(rr[0]), u2 = u01(rr[1]);
  const double h = 1.0 / P.dt;
  double wt;
  bool killed;
  if (P.rb_weight) {
    // E[min(T1, T2)] = 1 / (h + k) and P(killed) = k / (h + k), k = k0 / p
    killed = u2 * (h * r.p + P.k0) < P.k0;
    wt = r.p / (h * r.p + P.k0);
  } else {
    double t1 = -std::log(1.0 - u1) / h;
    double t2 = -std::log(1.0 - u2) * r.p / P.k0;
    killed = !(t1 < t2);
    wt = killed ? t2 : t1;
  }
  rec.killed = killed;
  for (int c = 0; c < 3; ++c) { rec.f[c] = r.f[c]; rec.val[c] = wt * r.f[c] / r.p; }
  rec.p = r.p;
  rec.pix = r.pix;
  rec.info = r.info;
  if (!killed) {
    if (P.drift_mode == D_FD) fd_score(T, x, P.eps, P.fd_h, score);
    else if (exact) for (int i = 0; i < d; ++i) score[i] = g[i];
    else std::fill(score, score + d, 0.0);
  } else {
    std::fill(score, score + d, 0.0);
  }
}

// The hold/kill clock of Accumulate (Alg. 1) for a state with density p:
// killed flag and splat weight (the race, or its Rao-Blackwellised form).
void clock(const Params& P, const Stream& st, uint32_t step, uint32_t chain, double p, bool* killed, double* wt) {
  uint32_t rr[4];
  st.draw(step, chain, 0, P_CLOCK, rr);
  const double u1 = u01(rr[0]), u2 = u01(rr[1]);
  const double h = 1.0 / P.dt;
  if (P.rb_weight) {
    *killed = u2 * (h * p + P.k0) < P.k0;
    *wt = p / (h * p + P.k0);
  } else {
    const double t1 = -std::log(1.0 - u1) / h;
    const double t2 = -std::log(1.0 - u2) * p / P.k0;
    *killed = !(t1 < t2);
    *wt = *killed ? t2 : t1;
  }
}

// MALA Restore (the paper's comparison method of Sec. 6 and App. A: Jump
// Restore whose local dynamics is a Metropolis-adjusted Langevin move, so the
// local kernel is pi-invariant and the killing rate k0 / p is the invariant
// one of Eq. invariant-killing-rate).  One move from x (current state, its
// record in rec and its score in score): the Langevin proposal
// y = x + (stddev^2 / 2) s(x) + stddev xi (the normals of Alg. 4, no rotation:
// the adjusted move is reversible), wrapped; accepted with probability
// min(1, p(y) q(x | y) / (p(x) q(y | x))),
// q(y | x) proportional to exp(-|y - x - (stddev^2 / 2) s(x)|^2 / (2 stddev^2))
// with torus differences to the nearest image.  Then the clock at the
// resulting state.
void mala_move(const Target& T, const Params& P, const Stream& st, uint32_t step, uint32_t chain, double* x,
               double* score, ChainRec& rec) {
  const int d = T.d();
  const double a = 0.5 * P.stddev * P.stddev;
  std::vector<double> y(x, x + d), sy(d, 0.0);
  for (int q = 0; q < d / 2; ++q) {
    uint32_t rr[4];
    st.draw(step, chain, (uint32_t)(q >> 1), P_NORMAL, rr);
    double ua = u01(rr[(q & 1) * 2]), ub = u01(rr[(q & 1) * 2 + 1]);
    double rad = std::sqrt(-2.0 * std::log(1.0 - ua));
    double th = 2.0 * PI * ub;
    y[2 * q] = wrap01(x[2 * q] + a * score[2 * q] + P.stddev * rad * std::cos(th));
    y[2 * q + 1] = wrap01(x[2 * q + 1] + a * score[2 * q + 1] + P.stddev * rad * std::sin(th));
  }
  EvalResult ry;
  evaluate(T, y.data(), P.eps, ry, sy.data());
  double fwd = 0.0, rev = 0.0;  // |y - x - a s(x)|^2 and |x - y - a s(y)|^2
  for (int i = 0; i < d; ++i) {
    double e1 = y[i] - x[i];
    e1 -= std::nearbyint(e1);
    e1 -= a * score[i];
    double e2 = x[i] - y[i];
    e2 -= std::nearbyint(e2);
    e2 -= a * sy[i];
    fwd += e1 * e1;
    rev += e2 * e2;
  }
  const double log_alpha = std::log(ry.p) - std::log(rec.p) + (fwd - rev) / (2.0 * P.stddev * P.stddev);
  uint32_t rr[4];
  st.draw(step, chain, 0, P_MH, rr);
  if (u01(rr[0]) < std::exp(log_alpha)) {
    std::copy(y.begin(), y.end(), x);
    std::copy(sy.begin(), sy.end(), score);
    for (int c = 0; c < 3; ++c) rec.f[c] = ry.f[c];
    rec.p = ry.p;
    rec.pix = ry.pix;
    rec.info = ry.info;
  }
  double wt;
  bool killed;
  clock(P, st, step, chain, rec.p, &killed, &wt);
  rec.killed = killed;
  for (int c = 0; c < 3; ++c) rec.val[c] = wt * rec.f[c] / rec.p;
}

// LocalDynamics (Alg. 4): for each coordinate pair,
// x += (stddev^2 / 2) s + gamma_tilde (s_2, -s_1) + stddev xi, then wrap.
void local_dynamics(const Params& P, const Stream& st, uint32_t step, uint32_t chain, int d, double* x,
                    const double* s) {
  const double a = 0.5 * P.stddev * P.stddev;
  for (int q = 0; q < d / 2; ++q) {
    uint32_t rr[4];
    st.draw(step, chain, (uint32_t)(q >> 1), P_NORMAL, rr);
    double ua = u01(rr[(q & 1) * 2]), ub = u01(rr[(q & 1) * 2 + 1]);
    double rad = std::sqrt(-2.0 * std::log(1.0 - ua));
    double th = 2.0 * PI * ub;
    double xi0 = rad * std::cos(th), xi1 = rad * std::sin(th);
    double s0 = s[2 * q], s1 = s[2 * q + 1];
    x[2 * q] = wrap01(x[2 * q] + a * s0 + P.gamma_tilde * s1 + P.stddev * xi0);
    x[2 * q + 1] = wrap01(x[2 * q + 1] + a * s1 - P.gamma_tilde * s0 + P.stddev * xi1);
  }
}

void regenerate(const Stream& st, uint32_t step, uint32_t chain, int d, double* x) {
  for (int i = 0; i < d; i += 4) {
    uint32_t rr[4];
    st.draw(step, chain, (uint32_t)(i >> 2), P_REGEN, rr);
    for (int k = 0; k < 4 && i + k < d; ++k) x[i + k] = u01(rr[k]);
  }
}

}  // namespace

// ====================================================================== C API
extern "C" {

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void* orc_scene_create(const float* verts, int nv, const int* tris, const float* normals, int nt,
                       const int* tri_mat, const float* mats, int nm, const float* cam, int W, int H,
                       int use_bvh) {
  (void)nv;
  Scene* S = new Scene();
  S->W = W;
  S->H = H;
  S->use_bvh = use_bvh != 0;
  for (int i = 0; i < nm; ++i) {
    const float* m = mats + 12 * i;
    Mat q;
    q.type = (int)m[0];
    for (int c = 0; c < 3; ++c) { q.albedo[c] = m[1 + c]; q.emit[c] = m[6 + c]; }
    q.rough = m[4];
    q.ior = m[5];
    q.f0 = m[9];
    for (int c = 0; c < 3; ++c) q.k[c] = m[9 + c];
    S->mats.push_back(q);
  }
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  auto V = [&](int i) { return D3(verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]); };
  auto Nrm = [&](int i) { return D3(normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]); };
  for (int i = 0; i < nt; ++i) {
    Tri t;
    t.v0 = V(tris[3 * i]); t.v1 = V(tris[3 * i + 1]); t.v2 = V(tris[3 * i + 2]);
    t.e1 = t.v1 - t.v0; t.e2 = t.v2 - t.v0;
    t.N = cross(t.e1, t.e2);
    double nn = dot(t.N, t.N);
    t.area = 0.5 * std::sqrt(nn);
    t.ng = t.N * (1.0 / std::sqrt(nn));
    t.au = cross(t.e2, t.N) * (1.0 / nn);
    t.av = cross(t.N, t.e1) * (1.0 / nn);
    t.mat = tri_mat[i];
    // shading normals only where all three vertex normals are non-zero
    t.has_n = false;
    if (normals) {
      t.n0 = Nrm(tris[3 * i]); t.n1 = Nrm(tris[3 * i + 1]); t.n2 = Nrm(tris[3 * i + 2]);
      t.has_n = dot(t.n0, t.n0) > 0.0 && dot(t.n1, t.n1) > 0.0 && dot(t.n2, t.n2) > 0.0;
    }
    const D3 vs[3] = {t.v0, t.v1, t.v2};
    for (int j = 0; j < 3; ++j) {
      const double c[3] = {vs[j].x, vs[j].y, vs[j].z};
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], c[a]); hi[a] = std::max(hi[a], c[a]); }
    }
    S->tris.push_back(t);
  }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  S->tmin = 1e-5 * ext;
  // lights: emissive triangles, selected with probability ~ area * lum(emission)
  S->sel.assign(nt, 0.0);
  double tot = 0.0;
  std::vector<double> pw;
  for (int i = 0; i < nt; ++i) {
    const Mat& m = S->mats[S->tris[i].mat];
    if (!m.emissive()) continue;
    double p = S->tris[i].area * (LUM[0] * m.emit[0] + LUM[1] * m.emit[1] + LUM[2] * m.emit[2]);
    if (!(p > 0)) continue;
    S->lights.push_back(i);
    pw.push_back(p);
    tot += p;
  }
  double acc = 0.0;
  for (size_t k = 0; k < S->lights.size(); ++k) {
    acc += pw[k];
    S->light_cdf.push_back(acc / tot);
    S->sel[S->lights[k]] = pw[k] / tot;
  }
  if (!S->light_cdf.empty()) S->light_cdf.back() = 1.0;
  // camera
  D3 eye(cam[0], cam[1], cam[2]), look(cam[3], cam[4], cam[5]), up(cam[6], cam[7], cam[8]);
  S->cam.eye = eye;
  S->cam.fwd = normalize(look - eye);
  S->cam.right = normalize(cross(S->cam.fwd, up));
  S->cam.up = cross(S->cam.right, S->cam.fwd);
  double th = std::tan(0.5 * cam[9] * PI / 180.0);
  S->cam.ty = th;
  S->cam.tx = th * (double)W / (double)H;
  if (S->use_bvh) build_bvh(*S);
  return S;
}

void orc_scene_destroy(void* s) { delete static_cast<Scene*>(s); }

int orc_scene_num_lights(void* s) { return (int)static_cast<Scene*>(s)->lights.size(); }

void* orc_mixture_create(int d, int K, const double* w, const double* mu, const double* sig, int W, int H,
                         double cval) {
  Mixture* M = new Mixture();
  M->d = d; M->K = K; M->W = W; M->H = H; M->cval = cval;
  M->w.assign(w, w + K);
  M->mu.assign(mu, mu + (size_t)K * d);
  M->sig.assign(sig, sig + K);
  return M;
}
void orc_mixture_destroy(void* m) { delete static_cast<Mixture*>(m); }

void* orc_step_create(int d, double c1, double c2, double w, int W, int H) {
  return new StepDensity{d, W, H, c1, c2, w};
}
void orc_step_destroy(void* p) { delete static_cast<StepDensity*>(p); }

// The bias term of Sec. 5.2 / App. C for a target on T^2 (d = 2):
// (L* p / p)(y) = h ((K* p)(y) / p(y) - 1), where L f = h (K f - f) is the
// generator of the continuous-time embedding of the local dynamics with
// holding rate h = 1 / dt (Sec. 4, Eq. diffusion-restore-holding-rate),
// K(x, .) is the Euler-Maruyama kernel of Alg. 4 (mean
// x + (stddev^2 / 2) s(x) + gamma_tilde J s(x), covariance stddev^2 I,
// wrapped on the torus; s = grad log p), and
// (K* p)(y) = int p(x) K(x, y) dx.  The integral is the trapezoid rule on
// the square of half-width `radius` * stddev around y with `n` nodes per
// side, each node's Gaussian summed over the nearest torus images.
// prm: stddev, dt, gamma_tilde, eps.  y [M * 2] -> out [M].
int orc_lstar_over_p(void* tgt, int kind, const double* prm, const double* y, int64_t M, double radius, int n,
                     double* out) {
  Target T = make_target(tgt, kind, 1);
  if (T.d() != 2 || n < 2) return -1;
  const double stddev = prm[0], dt = prm[1], gt = prm[2], eps = prm[3];
  const double a = 0.5 * stddev * stddev, h = 1.0 / dt;
  const double half = radius * stddev, dx = 2.0 * half / (n - 1);
  const double norm = 1.0 / (2.0 * PI * stddev * stddev);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t m = 0; m < M; ++m) {
    const double y0 = y[2 * m], y1 = y[2 * m + 1];
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      const double wi = (i == 0 || i == n - 1) ? 0.5 : 1.0;
      for (int j = 0; j < n; ++j) {
        const double wj = (j == 0 || j == n - 1) ? 0.5 : 1.0;
        double x[2] = {y0 - half + i * dx, y1 - half + j * dx};
        EvalResult r;
        double s[2];
        evaluate(T, x, eps, r, s);
        // mean of the kernel from x, and its offset to y (nearest image)
        double e0 = y0 - (x[0] + a * s[0] + gt * s[1]);
        double e1 = y1 - (x[1] + a * s[1] - gt * s[0]);
        e0 -= std::nearbyint(e0);
        e1 -= std::nearbyint(e1);
        acc += wi * wj * r.p * norm * std::exp(-0.5 * (e0 * e0 + e1 * e1) / (stddev * stddev));
      }
    }
    EvalResult ry;
    double yy[2] = {y0, y1};
    evaluate(T, yy, eps, ry, nullptr);
    out[m] = h * (acc * dx * dx / ry.p - 1.0);
  }
  return 0;
}

// Closest-hit queries: tri = -1 on miss.
void orc_trace(void* s, const double* o, const double* d, int64_t n, int exclude, int* tri, double* t,
               long* tests) {
  Scene* S = static_cast<Scene*>(s);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int tr = -1;
    double th = INFINITY;
    long cnt = 0;
    if (!closest(*S, D3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), D3(d[3 * i], d[3 * i + 1], d[3 * i + 2]), exclude,
                 &tr, &th, &cnt)) tr = -1;
    tri[i] = tr;
    t[i] = th;
    if (tests) tests[i] = cnt;
  }
}

// Batched evaluation of f, log p (p = lum f + eps), the pixel, and optionally
// grad log p (forward-mode duals).  info (nullable): per point 4 * 20 ints
// (tri, lobe, vis, light per vertex) + nseg + rays.
enum { INFO_STRIDE = 4 * PathInfo::MAXV + 2 };
int orc_info_stride() { return INFO_STRIDE; }

static void pack_info(const PathInfo& pi, int* o) {
  for (int v = 0; v < PathInfo::MAXV; ++v) {
    o[v] = pi.tri[v];
    o[PathInfo::MAXV + v] = pi.lobe[v];
    o[2 * PathInfo::MAXV + v] = pi.vis[v];
    o[3 * PathInfo::MAXV + v] = pi.light[v];
  }
  o[4 * PathInfo::MAXV] = pi.nseg;
  o[4 * PathInfo::MAXV + 1] = pi.rays;
}

int orc_eval(void* tgt, int kind, int L, const double* x, int64_t M, double eps, double* f, double* logp,
             double* grad, int* pix, int* info) {
  Target T = make_target(tgt, kind, L);
  const int d = T.d();
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < M; ++i) {
    EvalResult r;
    evaluate(T, x + i * d, eps, r, grad ? grad + i * d : nullptr);
    if (f) for (int c = 0; c < 3; ++c) f[3 * i + c] = r.f[c];
    if (logp) logp[i] = std::log(r.p);
    if (pix) pix[i] = r.pix;
    if (info) pack_info(r.info, info + i * INFO_STRIDE);
  }
  return 0;
}

int orc_fd_score(void* tgt, int kind, int L, const double* x, int64_t M, double eps, double h, double* score) {
  Target T = make_target(tgt, kind, L);
  const int d = T.d();
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < M; ++i) fd_score(T, x + i * d, eps, h, score + i * d);
  return 0;
}

// BSDF unit access (tests).  mat: 12 floats.  n, wo: unit vectors.
int orc_bsdf_sample(const float* mat, const double* n, const double* wo, double u1, double u2, double* wi,
                    double* w, double* pdf, int* lobe) {
  Mat m;
  m.type = (int)mat[0];
  for (int c = 0; c < 3; ++c) { m.albedo[c] = mat[1 + c]; m.emit[c] = mat[6 + c]; }
  m.rough = mat[4]; m.ior = mat[5]; m.f0 = mat[9];
  for (int c = 0; c < 3; ++c) m.k[c] = mat[9 + c];
  D3 N(n[0], n[1], n[2]), WO(wo[0], wo[1], wo[2]), WI;
  double ww[3], pp;
  int lb = -1;
  bool ok = opaque_sample<double>(m, N, N, WO, u1, u2, WI, ww, pp, lb);
  wi[0] = WI.x; wi[1] = WI.y; wi[2] = WI.z;
  for (int c = 0; c < 3; ++c) w[c] = ok ? ww[c] : 0.0;
  *pdf = ok ? pp : 0.0;
  *lobe = lb;
  return ok ? 1 : 0;
}

void orc_bsdf_eval(const float* mat, const double* n, const double* wo, const double* wi, double* fs, double* pdf) {
  Mat m;
  m.type = (int)mat[0];
  for (int c = 0; c < 3; ++c) { m.albedo[c] = mat[1 + c]; m.emit[c] = mat[6 + c]; }
  m.rough = mat[4]; m.ior = mat[5]; m.f0 = mat[9];
  for (int c = 0; c < 3; ++c) m.k[c] = mat[9 + c];
  D3 N(n[0], n[1], n[2]), WO(wo[0], wo[1], wo[2]), WI(wi[0], wi[1], wi[2]);
  bsdf_eval<double>(m, N, WO, WI, fs, *pdf);
}

double orc_fresnel_dielectric(double ci, double ct, double eta) { return fresnel_dielectric(ci, ct, eta); }
double orc_fresnel_conductor(double ci, double eta, double k) { return fresnel_conductor<double>(ci, eta, k); }

// One Evolve move of x (Alg. 2 / Alg. 4) for a surviving chain, given score;
// exposes the LocalDynamics step alone for closed-form checks.
void orc_local_dynamics(const double* prm, uint64_t seed, uint32_t frame, uint32_t step, uint32_t chain, int d,
                        const double* x, const double* score, double* xo) {
  Params P{};
  P.stddev = prm[0];
  P.gamma_tilde = prm[1];
  Stream st{{(uint32_t)seed, (uint32_t)(seed >> 32)}, frame};
  std::copy(x, x + d, xo);
  local_dynamics(P, st, step, chain, d, xo, score);
}

// Runs Restore chains (Alg. 1 at step 0, then n_steps calls of Alg. 2).
// chain_ids[M]: the chain indices (each chain's Philox stream depends only
// on (seed, frame, chain, step)).  Per-step outputs are optional (nullable);
// each is laid out [n_steps + 1][M][...].  accum (nullable, W*H*3) receives
// the splat values summed in FP64 in (step, chain) order; tour_count the
// number of kills; p_init_sum the sum of p over the init pass (for
// p_lambda = sum / M).
int orc_restore_run(void* tgt, int kind, const Params* prm, uint64_t seed, uint32_t frame,
                    const uint32_t* chain_ids, int64_t M, int n_steps, double* x_out, double* logp_out,
                    double* score_out, uint8_t* killed_out, int* pix_out, double* val_out, int* info_out,
                    double* accum, uint64_t* tour_count, double* p_init_sum) {
  Target T = make_target(tgt, kind, prm->L);
  const Params P = *prm;
  const int d = T.d();
  const int WH = T.W() * T.H();
  Stream st{{(uint32_t)seed, (uint32_t)(seed >> 32)}, frame};
  std::vector<double> X((size_t)M * d), S((size_t)M * d, 0.0);
  std::vector<uint8_t> K(M, 0);
  std::vector<ChainRec> R(M);
  uint64_t tours = 0;
  double psum = 0.0;
  for (int s = 0; s <= n_steps; ++s) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < M; ++j) {
      const uint32_t c = chain_ids[j];
      double* x = X.data() + j * d;
      double* sc = S.data() + j * d;
      if (s == 0 || K[j]) {
        regenerate(st, (uint32_t)s, c, d, x);
        accumulate(T, P, st, (uint32_t)s, c, x, sc, R[j]);
      } else if (P.drift_mode == D_MALA) {
        mala_move(T, P, st, (uint32_t)s, c, x, sc, R[j]);
      } else {
        local_dynamics(P, st, (uint32_t)s, c, d, x, sc);
        accumulate(T, P, st, (uint32_t)s, c, x, sc, R[j]);
      }
      K[j] = R[j].killed ? 1 : 0;
    }
    for (int64_t j = 0; j < M; ++j) {
      const ChainRec& r = R[j];
      tours += r.killed ? 1 : 0;
      if (s == 0) psum += r.p;
      if (accum) for (int c = 0; c < 3; ++c) accum[(size_t)r.pix * 3 + c] += r.val[c];
      const size_t o = (size_t)s * M + j;
      if (x_out) std::copy(X.begin() + j * d, X.begin() + (j + 1) * d, x_out + o * d);
      if (score_out) std::copy(S.begin() + j * d, S.begin() + (j + 1) * d, score_out + o * d);
      if (logp_out) logp_out[o] = std::log(r.p);
      if (killed_out) killed_out[o] = K[j];
      if (pix_out) pix_out[o] = r.pix;
      if (val_out) for (int c = 0; c < 3; ++c) val_out[o * 3 + c] = r.val[c];
      if (info_out) pack_info(r.info, info_out + o * INFO_STRIDE);
    }
  }
  (void)WH;
  if (tour_count) *tour_count = tours;
  if (p_init_sum) *p_init_sum = psum;
  return 0;
}

// Complete tours (Sec. 4.3: a tour is one local exploration up to its
// termination).  Chain j starts at a regeneration (x ~ U(T^d), step 0) and
// runs Alg. 2 until its first kill, or until max_steps steps (then flagged
// as truncated).  Tours are i.i.d., so by the renewal-reward theorem the
// long-run time average of g equals E[int_tour g] / E[int_tour 1], and the
// Restore image is k0 / #tours * sum over tours of int_tour f / p.
// Outputs per tour: I1 = sum of weights, Ix[d] = sum of weight * x,
// Ixx[d*d] = sum of weight * x x^T, steps, truncated; accum (nullable,
// W*H*3) receives sum of weight * f / p over all tours.
int orc_restore_tours(void* tgt, int kind, const Params* prm, uint64_t seed, uint32_t frame,
                      const uint32_t* chain_ids, int64_t M, int64_t max_steps, double* I1, double* Ix, double* Ixx,
                      int64_t* steps, uint8_t* truncated, double* accum) {
  Target T = make_target(tgt, kind, prm->L);
  const Params P = *prm;
  const int d = T.d();
  const size_t npix = (size_t)T.W() * T.H();
  Stream st{{(uint32_t)seed, (uint32_t)(seed >> 32)}, frame};
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<std::vector<double>> acc_t(accum ? nth : 0, std::vector<double>(accum ? npix * 3 : 0, 0.0));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < M; ++j) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    const uint32_t c = chain_ids[j];
    std::vector<double> x(d), sc(d, 0.0);
    double i1 = 0.0;
    std::vector<double> ix(d, 0.0), ixx((size_t)d * d, 0.0);
    ChainRec r;
    int64_t s = 0;
    bool done = false;
    for (; s <= max_steps; ++s) {
      if (s == 0) {
        regenerate(st, 0, c, d, x.data());
        accumulate(T, P, st, 0, c, x.data(), sc.data(), r);
      } else if (P.drift_mode == D_MALA) {
        mala_move(T, P, st, (uint32_t)s, c, x.data(), sc.data(), r);
      } else {
        local_dynamics(P, st, (uint32_t)s, c, d, x.data(), sc.data());
        accumulate(T, P, st, (uint32_t)s, c, x.data(), sc.data(), r);
      }
      // the splat weight (hold time, or its Rao-Blackwellised mean)
      uint32_t rr[4];
      st.draw((uint32_t)s, c, 0, P_CLOCK, rr);
      double wt;
      if (P.rb_weight) {
        wt = r.p / ((1.0 / P.dt) * r.p + P.k0);
      } else {
        const double t1 = -std::log(1.0 - u01(rr[0])) * P.dt;
        const double t2 = -std::log(1.0 - u01(rr[1])) * r.p / P.k0;
        wt = r.killed ? t2 : t1;
      }
      i1 += wt;
      for (int a = 0; a < d; ++a) {
        ix[a] += wt * x[a];
        for (int b = 0; b < d; ++b) ixx[(size_t)a * d + b] += wt * x[a] * x[b];
      }
      if (accum) for (int k = 0; k < 3; ++k) acc_t[tid][(size_t)r.pix * 3 + k] += r.val[k];
      if (r.killed) { done = true; break; }
    }
    I1[j] = i1;
    for (int a = 0; a < d; ++a) Ix[j * d + a] = ix[a];
    for (size_t q = 0; q < (size_t)d * d; ++q) Ixx[(size_t)j * d * d + q] = ixx[q];
    steps[j] = done ? s + 1 : s;
    truncated[j] = done ? 0 : 1;
  }
  if (accum)
    for (int t = 0; t < nth; ++t)
      for (size_t q = 0; q < npix * 3; ++q) accum[q] += acc_t[t][q];
  return 0;
}

// Ordinary Monte Carlo (path tracing) over the same f: per pixel, spp
// samples with the film pair stratified to the pixel and the other
// coordinates uniform.  mean/var (W*H*3): per-pixel sample mean of f / (W H)
// and the variance of that mean.
int orc_pt_image(void* s, int L, int spp, uint64_t seed, double* mean, double* var) {
  Scene* S = static_cast<Scene*>(s);
  const int d = 2 + 4 * (L - 1);
  const int W = S->W, H = S->H;
  Stream st{{(uint32_t)seed, (uint32_t)(seed >> 32)}, 0};
  const double WH = (double)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int pix = 0; pix < W * H; ++pix) {
    int row = pix / W, col = pix % W;
    std::vector<double> x(d);
    double m1[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
    for (int k = 0; k < spp; ++k) {
      for (int i = 0; i < d; i += 4) {
        uint32_t rr[4];
        st.draw((uint32_t)k, (uint32_t)pix, (uint32_t)(i >> 2), P_PT, rr);
        for (int q = 0; q < 4 && i + q < d; ++q) x[i + q] = u01(rr[q]);
      }
      x[0] = (col + x[0]) / W;
      x[1] = (row + x[1]) / H;
      PathOut<double> po;
      eval_path(*S, x.data(), L, po);
      for (int c = 0; c < 3; ++c) { double v = po.f[c] / WH; m1[c] += v; m2[c] += v * v; }
    }
    for (int c = 0; c < 3; ++c) {
      double mu = m1[c] / spp;
      mean[pix * 3 + c] = mu;
      var[pix * 3 + c] = std::max(0.0, m2[c] / spp - mu * mu) / spp;
    }
  }
  return 0;
}

}  // extern "C"
