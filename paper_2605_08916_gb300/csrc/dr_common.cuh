// Device-side basics for the Diffusion Restore CUDA library (sm_103a):
// float3 arithmetic, the Philox4x32-10 counter-based generator and its
// uniform / normal conversions, and the HBM layouts shared by the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define DR_HD __host__ __device__ __forceinline__
#define DR_D __device__ __forceinline__

namespace dr {

constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kLumR = 0.2126f, kLumG = 0.7152f, kLumB = 0.0722f;
constexpr int kMaxPathLen = 16;               // L <= 16  ->  d <= 62
// Entries of the per-thread traversal stack; a BVH deeper than this + 1 is
// rejected at scene upload.
constexpr int kTraversalStack = 48;
// entries of the two-level walk's stack (a TLAS path, a return mark and a
// BLAS path); its kernels get the larger shared-memory stack
constexpr int kTraversalStackTL = 64;
constexpr int kMaxDim = 2 + 4 * (kMaxPathLen - 1);

// device error word bits (read back by the host after each call)
enum : uint32_t {
  kErrStackOverflow = 1u << 0,
  kErrNonFinite = 1u << 1,
  kErrBadIndex = 1u << 2,
  kErrTimeout = 1u << 3,
};

// ------------------------------------------------------------------ float3
DR_HD float3 f3(float a, float b, float c) { return make_float3(a, b, c); }
DR_HD float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
DR_HD float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
DR_HD float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
DR_HD float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
DR_HD float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
DR_HD float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
DR_HD float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
DR_HD float3& operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
DR_HD float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
DR_HD float3 cross(float3 a, float3 b) { return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
DR_HD float lum(float3 c) { return kLumR * c.x + kLumG * c.y + kLumB * c.z; }
DR_HD float3 lum_weights() { return f3(kLumR, kLumG, kLumB); }
DR_D float3 normalize(float3 a) { return a * rsqrtf(dot(a, a)); }
DR_D float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

// Backward of y = a / |a| given dy: returns da.
DR_D float3 normalize_bwd(float3 a_unnorm, float3 y, float3 dy) {
  float inv = rsqrtf(dot(a_unnorm, a_unnorm));
  return (dy - y * dot(y, dy)) * inv;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with the round multipliers, a word permutation
// with xors of the key, and a Weyl bump of the key between rounds.
struct U4 { uint32_t a, b, c, d; };

DR_HD U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Stream identity: key = (seed_lo, seed_hi); counter = (step, chain, block,
// frame << 4 | purpose).
enum Purpose : uint32_t { kRegen = 0, kNormal = 1, kClock = 2, kPT = 3, kMH = 4 };

struct Rng {
  uint32_t k0, k1, frame;
  DR_D U4 draw(uint32_t step, uint32_t chain, uint32_t block, uint32_t purpose) const {
    return philox4x32_10(step, chain, block, (frame << 4) | purpose, k0, k1);
  }
};

// 24-bit uniform in [0, 1): exact in float.
DR_HD float u01(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

// Box-Muller pair from two uniforms (u in [0,1) so 1 - u in (0, 1]).
DR_D float2 box_muller(float ua, float ub) {
  const float r = sqrtf(-2.0f * logf(1.0f - ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  return make_float2(r * c, r * s);
}

// Torus wrap x - floor(x); a result that rounds to 1 becomes 0.
DR_D float wrap01(float v) {
  const float r = v - floorf(v);
  return r >= 1.0f ? 0.0f : r;
}

// ------------------------------------------------------------------ layouts
// BVH node (64 B, 4 x float4): both children's boxes live in the parent.
//   n0 = (c0.lo.x, c0.lo.y, c0.lo.z, c0.hi.x)
//   n1 = (c0.hi.y, c0.hi.z, c1.lo.x, c1.lo.y)
//   n2 = (c1.lo.z, c1.hi.x, c1.hi.y, c1.hi.z)
//   n3 = (child0, child1, -, -) as ints; child >= 0: inner node index;
//        child < 0: leaf, first = (child & 0x7fffffff) >> 3, count = (child & 7) + 1
// Triangle (48 B, 3 x float4) in leaf order:
//   t0 = (v0, orig id as int bits), t1 = (e1 = v1 - v0, -), t2 = (e2 = v2 - v0, -)
// Surface record per original triangle (80 B, 5 x float4), used for shading
// and the differentiable hit point:
//   s0 = (v0, material id bits), s1 = (N = cross(e1, e2), area), s2 = (ng, flags),
//   s3 = (au, -), s4 = (av, -) where barycentrics are (P - v0).au, (P - v0).av
// Light record (64 B, 4 x float4): l0 = (v0, tri id bits), l1 = (v1, selection
// probability), l2 = (v2, area), l3 = (cdf upper bound, emission rgb of the
// triangle's material).
// Material: 12 floats [type, albedo rgb, roughness, ior, emission rgb, f0, -, -];
// a conductor keeps the real part eta of its complex index (RGB) in the
// albedo slots and the imaginary part k (RGB) in the last three.
constexpr int kNodeF4 = 4, kTriF4 = 3, kSurfF4 = 5, kLightF4 = 4, kMatFloats = 12;
enum MatType { kDiffuse = 0, kGlossy = 1, kDielectric = 2, kEmitter = 3, kConductor = 4 };
constexpr float kGlossySpecProb = 0.5f;

// 4-wide BVH node (112 B, 7 x float4): lo.x[4], hi.x[4], lo.y[4], hi.y[4],
// lo.z[4], hi.z[4], then the four child links (inner index, leaf code, or
// kBvh4Empty, whose box is inverted: lo = +inf, hi = -inf); leaves hold up
// to kBvh4MaxLeaf triangles.
constexpr int kNode4F4 = 7;
constexpr int kBvh4MaxLeaf = 4;
constexpr int kBvh4Empty = 0x7fffffff;

// 8-wide compressed BVH node (80 B, 5 x uint4), child boxes quantised to
// 8 bits per plane against the node's own box:
//   w0 = (p.x, p.y, p.z as float bits, ex | ey << 8 | ez << 16 | imask << 24)
//        with signed 8-bit exponents e: a child's box is
//        [p + 2^e * qlo, p + 2^e * qhi] per axis (never smaller than the
//        child's exact box)
//   w1 = (child_base, tri_base, meta[0..3], meta[4..7])
//   w2 = (qlo.x[0..3], qlo.x[4..7], qlo.y[0..3], qlo.y[4..7])
//   w3 = (qlo.z[0..3], qlo.z[4..7], qhi.x[0..3], qhi.x[4..7])
//   w4 = (qhi.y[0..3], qhi.y[4..7], qhi.z[0..3], qhi.z[4..7])
// Slot s holds an inner child if bit s of imask is set: node child_base +
// popc(imask & ((1 << s) - 1)) (a node's inner children are consecutive);
// a leaf if bit 7 of meta[s] is set: triangles tri_base + (meta & 31) ..
// + ((meta >> 5) & 3) (at most kBvh4MaxLeaf); else the slot is empty.
// Children sit in slots by the octant heuristic: rays whose direction signs
// form octant o (bit 0: x < 0, bit 1: y < 0, bit 2: z < 0) visit slot k ^ o
// k-th, which roughly orders them near to far.
constexpr int kNode8U4 = 5;

// Two-level BVH of an instanced scene: a 4-wide TLAS over the instances'
// world boxes whose leaves hold one instance each (leaf first = instance
// index), and the meshes' 4-wide BLASes concatenated (inner links and leaf
// ranges global in the concatenation; triangle records in object space,
// t0.w = the triangle's index within its mesh).  Instance record (64 B,
// 4 x float4): rows 0..2 of the world-to-object affine map as (m0, m1, m2,
// c) so that p_obj = (m . p_world) + c per row, then (BLAS root node, global
// id of the instance's first triangle, -, -) as int bits.
constexpr int kInstF4 = 4;

DR_HD int leaf_code(int first, int count) { return (int)(0x80000000u | ((uint32_t)first << 3) | (uint32_t)(count - 1)); }
DR_HD int leaf_first(int c) { return (int)(((uint32_t)c & 0x7fffffffu) >> 3); }
DR_HD int leaf_count(int c) { return (int)((uint32_t)c & 7u) + 1; }

// One splat record: pixel index and the RGB splat value dt * f / p.
struct __align__(16) SplatRec {
  uint32_t pix;
  float r, g, b;
};

struct Camera {
  float3 eye, fwd, right, up;
  float tx, ty;
};

struct DevScene {
  const float4* __restrict__ nodes;
  const float4* __restrict__ nodes4;  // 4-wide BVH (null: use the binary one)
  const float4* __restrict__ tris4;   // triangles in the 4-wide BVH's leaf order
  const uint4* __restrict__ nodes8;   // 8-wide compressed BVH (null: not built)
  const float4* __restrict__ tris8;   // triangles in the 8-wide BVH's leaf order
  const float4* __restrict__ tl_nodes;  // two-level BVH (null: not built): TLAS nodes (4-wide)
  const float4* __restrict__ bl_nodes;  // concatenated BLAS nodes (4-wide)
  const float4* __restrict__ bl_tris;   // concatenated BLAS triangles (object space)
  const float4* __restrict__ insts;     // instance records
  int n_tl_nodes, n_bl_nodes, n_bl_tris, n_insts;
  const float4* __restrict__ tris;
  const float4* __restrict__ surf;
  const float* __restrict__ nrm;     // 9 floats per original triangle, or null
  const float* __restrict__ mats;
  const float4* __restrict__ lights;
  int n_lights, n_tris, n_nodes, n_nodes4, n_nodes8, W, H;
  float tmin;
  Camera cam;
};

// Analytic target: isotropic Gaussian mixture on the torus (K = 0: constant).
struct DevMixture {
  const float* __restrict__ w;    // K
  const float* __restrict__ mu;   // K * d
  const float* __restrict__ sig;  // K
  int K, d, W, H;
  float cval;
};

}  // namespace dr
