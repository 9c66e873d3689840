// BVH traversal for the path-contribution kernels.
//
// The paper traces rays with hardware RT cores through a graphics API
// (Sec. 4.3, "ray tracing and compute shaders"); GB300 has no RT cores, so
// traversal is software: a binary BVH whose nodes hold both children's boxes
// (one 64-B node = four 16-B vector loads), leaf triangles in 48-B records
// (three 16-B loads), read through the read-only path, and a per-thread
// traversal stack staged in shared memory (layout [depth][thread], so a warp's
// pushes and pops hit 32 distinct banks).
#pragma once
#include "dr_common.cuh"

namespace dr {

// Per-ray bound on inner-node visits: far above any legitimate traversal of
// the scenes here, it caps the time a corrupt hierarchy could take; hitting
// it sets kErrBadIndex.
constexpr int kMaxNodeVisits = 1 << 15;

struct Ray {
  float3 o, d, inv;
  float3 oinv;  // o * inv (rounded), for the 4-wide slab test
};

// A NaN in the ray makes every slab test pass (fminf / fmaxf drop NaNs), so
// such a ray would walk the whole tree: it is refused up front.
DR_D bool ray_finite(float3 o, float3 d) {
  return isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) && isfinite(d.z);
}

DR_D Ray make_ray(float3 o, float3 d) {
  Ray r;
  r.o = o;
  r.d = d;
  // a zero (or tiny) direction component gets a huge finite inverse rather
  // than an infinite one, so that no slab product is 0 * inf = NaN
  auto safe_inv = [](float v) { return 1.0f / (fabsf(v) > 1e-20f ? v : copysignf(1e-20f, v)); };
  r.inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
  r.oinv = f3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
  return r;
}

// Slab test of one box against [0, tmax]: the entry distance (>= 0) of a
// hit box, or -1 for a miss.  (A miss must not compare below an infinite
// tmax, so it is negative rather than +inf.)
// The differences lo - o are taken before scaling (not lo / d - o / d),
// which keeps the distances accurate when the origin lies far from the
// scene origin; the inverse is finite (see make_ray).
DR_D float box_entry(float3 lo, float3 hi, const Ray& r, float tmax) {
  const float tx0 = (lo.x - r.o.x) * r.inv.x, tx1 = (hi.x - r.o.x) * r.inv.x;
  const float ty0 = (lo.y - r.o.y) * r.inv.y, ty1 = (hi.y - r.o.y) * r.inv.y;
  const float tz0 = (lo.z - r.o.z) * r.inv.z, tz1 = (hi.z - r.o.z) * r.inv.z;
  const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  // a small relative slack keeps boxes of hits at exactly tmax
  return tn <= tf * 1.0000002f ? tn : -1.0f;
}

// Moller-Trumbore; hit iff det != 0, u >= 0, v >= 0, u + v <= 1, tmin < t < tmax.
DR_D bool tri_test(float3 v0, float3 e1, float3 e2, const Ray& r, float tmin, float tmax, float* t_out) {
  const float3 p = cross(r.d, e2);
  const float det = dot(e1, p);
  if (det == 0.0f) return false;
  // most candidates fail the barycentric bounds: they are rejected before
  // the division, on the numerators scaled by |det|; the survivors take the
  // exact test on the divided values
  const float sg = det < 0.0f ? -1.0f : 1.0f, adet = fabsf(det);
  const float3 tv = r.o - v0;
  const float du = dot(tv, p);
  if (du * sg < 0.0f || du * sg > adet) return false;
  const float3 q = cross(tv, e1);
  const float dv = dot(r.d, q);
  if (dv * sg < 0.0f || (du + dv) * sg > adet) return false;
  const float inv = 1.0f / det;
  const float u = du * inv;
  if (u < 0.0f || u > 1.0f) return false;
  const float v = dv * inv;
  if (v < 0.0f || u + v > 1.0f) return false;
  const float t = dot(e2, q) * inv;
  if (!(t > tmin && t < tmax)) return false;
  *t_out = t;
  return true;
}

struct TraceStats {
  uint32_t nodes, tris;
};

template <int STACK>
struct TraceStack {
  int* base;  // shared memory, [STACK][blockDim.x]
  int stride;
  DR_D int& at(int i) { return base[i * stride]; }
};

DR_D void load_node(const float4* __restrict__ nodes, int n, float3& lo0, float3& hi0, float3& lo1, float3& hi1,
                    int& c0, int& c1) {
  const float4 a = __ldg(nodes + 4 * n + 0);
  const float4 b = __ldg(nodes + 4 * n + 1);
  const float4 c = __ldg(nodes + 4 * n + 2);
  const int4 e = __ldg(reinterpret_cast<const int4*>(nodes) + 4 * n + 3);
  lo0 = f3(a.x, a.y, a.z);
  hi0 = f3(a.w, b.x, b.y);
  lo1 = f3(b.z, b.w, c.x);
  hi1 = f3(c.y, c.z, c.w);
  c0 = e.x;
  c1 = e.y;
}

DR_D float f4c(float4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
DR_D int i4c(int4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// Tests the triangles of one leaf against [tmin, tbest]; keeps the closest
// (ties: smaller original id).
// tris: the leaf-ordered triangle records of n_tris; id_base: added to each
// record's id (the instance's first global id in a BLAS, else 0).
template <bool STATS>
DR_D void leaf_closest_at(const float4* __restrict__ tris, int n_tris, int id_base, const DevScene& S, int code,
                          const Ray& r, int exclude, float& tbest, int& best, uint32_t* err, TraceStats* stats) {
  const int first = leaf_first(code);
  int cnt = leaf_count(code);
  if (first + cnt > n_tris) {
    *err |= kErrBadIndex;
    cnt = 0;
  }
  for (int i = 0; i < cnt; ++i) {
    const float4 t0 = __ldg(tris + 3 * (first + i) + 0);
    const float4 t1 = __ldg(tris + 3 * (first + i) + 1);
    const float4 t2 = __ldg(tris + 3 * (first + i) + 2);
    const int id = id_base + __float_as_int(t0.w);
    if (STATS) ++stats->tris;
    float th;
    if (id != exclude && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tbest * 1.0000001f + 1e-30f, &th)) {
      if (th < tbest || (th == tbest && id < best)) {
        tbest = th;
        best = id;
      }
    }
  }
}

template <bool STATS>
DR_D void leaf_closest(const DevScene& S, int code, const Ray& r, int exclude, float& tbest, int& best, uint32_t* err,
                       TraceStats* stats) {
  leaf_closest_at<STATS>(S.tris4, S.n_tris, 0, S, code, r, exclude, tbest, best, err, stats);
}

// Any hit among a leaf's triangles in (tmin, tmax), skipping two ids.
template <bool STATS>
DR_D bool leaf_any_at(const float4* __restrict__ tris, int n_tris, int id_base, const DevScene& S, int code,
                      const Ray& r, float tmax, int ex0, int ex1, uint32_t* err, TraceStats* stats) {
  const int first = leaf_first(code);
  int cnt = leaf_count(code);
  if (first + cnt > n_tris) {
    *err |= kErrBadIndex;
    cnt = 0;
  }
  for (int i = 0; i < cnt; ++i) {
    const float4 t0 = __ldg(tris + 3 * (first + i) + 0);
    const float4 t1 = __ldg(tris + 3 * (first + i) + 1);
    const float4 t2 = __ldg(tris + 3 * (first + i) + 2);
    const int id = id_base + __float_as_int(t0.w);
    if (STATS) ++stats->tris;
    float th;
    if (id != ex0 && id != ex1 && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tmax, &th)) return true;
  }
  return false;
}

// 4-wide traversal, one node per call so that a caller can interleave rays
// (the persistent trace passes refill finished lanes between steps).  The
// four child boxes of a node are tested together; leaves are tested on the
// spot, hit inner children are visited nearest first (the others pushed
// far-to-near).
struct Walk4 {
  int node, sp, budget;
};

// budget: every inner node and every leaf (at most four per node) once
DR_D Walk4 walk4_begin(const DevScene& S) { return Walk4{0, 0, min(5 * S.n_nodes4 + 64, kMaxNodeVisits)}; }

// Entry distances of a node's four child boxes against [0, tmax] (-1: a
// miss), and its links.  Per axis the ray's direction sign picks which slab
// plane is near, so no min / max pair is needed, and each distance is one
// fused multiply-add, plane * (1/d) - o * (1/d).  That form loses accuracy
// when the origin lies far from the scene origin (o/d is rounded), so the
// near distances subtract, and the far ones add, a margin of 2^-22 |o/d|
// (more than the rounding): boxes are only ever widened, never missed, and
// the closest hit is decided by the exact triangle tests.
DR_D void node4_entries_at(const float4* __restrict__ nodes, int node, const Ray& r, float tmax, float e[4],
                           int4& ch) {
  const float4* nb = nodes + (size_t)kNode4F4 * node;
  const int sx = r.inv.x < 0.0f, sy = r.inv.y < 0.0f, sz = r.inv.z < 0.0f;
  const float4 nx = __ldg(nb + sx), fx = __ldg(nb + 1 - sx);
  const float4 ny = __ldg(nb + 2 + sy), fy = __ldg(nb + 3 - sy);
  const float4 nz = __ldg(nb + 4 + sz), fz = __ldg(nb + 5 - sz);
  ch = __ldg(reinterpret_cast<const int4*>(nb + 6));
  constexpr float kM = 2.384185791015625e-07f;  // 2^-22
  const float onx = fmaf(fabsf(r.oinv.x), kM, r.oinv.x), ofx = fmaf(-fabsf(r.oinv.x), kM, r.oinv.x);
  const float ony = fmaf(fabsf(r.oinv.y), kM, r.oinv.y), ofy = fmaf(-fabsf(r.oinv.y), kM, r.oinv.y);
  const float onz = fmaf(fabsf(r.oinv.z), kM, r.oinv.z), ofz = fmaf(-fabsf(r.oinv.z), kM, r.oinv.z);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float tnx = fmaf(f4c(nx, k), r.inv.x, -onx), tfx = fmaf(f4c(fx, k), r.inv.x, -ofx);
    const float tny = fmaf(f4c(ny, k), r.inv.y, -ony), tfy = fmaf(f4c(fy, k), r.inv.y, -ofy);
    const float tnz = fmaf(f4c(nz, k), r.inv.z, -onz), tfz = fmaf(f4c(fz, k), r.inv.z, -ofz);
    const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.0f));
    const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tmax));
    e[k] = tn <= tf * 1.0000002f ? tn : -1.0f;
  }
}

DR_D void node4_entries(const DevScene& S, int node, const Ray& r, float tmax, float e[4], int4& ch) {
  node4_entries_at(S.nodes4, node, r, tmax, e, ch);
}

// A closest-hit walk's step at inner node w.node of `nodes`: hit children
// (leaves and inner nodes alike) nearest first, the nearest next, the
// others pushed far-to-near.  Returns true when the walk is over.
template <int STACK, bool STATS>
DR_D bool closest4_inner(const float4* __restrict__ nodes, const Ray& r, Walk4& w, float tbest, TraceStack<STACK> st,
                         uint32_t* err, TraceStats* stats) {
  int4 ch;
  float e[4];
  node4_entries_at(nodes, w.node, r, tbest, e, ch);
  if (STATS) ++stats->nodes;
  bool ok[4];
  int nc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // (an empty slot's inverted box is always a miss: e[k] < 0)
    ok[k] = e[k] >= 0.0f && e[k] <= tbest;
    nc += ok[k] ? 1 : 0;
  }
  if (nc == 0) {
    if (w.sp == 0) return true;
    w.node = st.at(--w.sp);
    return false;
  }
  if (w.sp + nc - 1 > STACK) {
    *err |= kErrStackOverflow;
    nc = STACK - w.sp + 1;
  }
  // near-to-far order by a five-exchange sorting network on (entry distance
  // bits, slot) keys; entries are >= 0 so their bit patterns sort like them
  uint32_t key[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) key[k] = ok[k] ? ((__float_as_uint(e[k]) & ~3u) | (uint32_t)k) : 0xffffffffu;
  auto cx = [](uint32_t& x, uint32_t& y) {
    const uint32_t lo = min(x, y), hi = max(x, y);
    x = lo;
    y = hi;
  };
  cx(key[0], key[1]);
  cx(key[2], key[3]);
  cx(key[0], key[2]);
  cx(key[1], key[3]);
  cx(key[1], key[2]);
  w.node = i4c(ch, (int)(key[0] & 3u));
#pragma unroll
  for (int i = 1; i < 4; ++i)
    if (i < nc) st.at(w.sp + nc - 1 - i) = i4c(ch, (int)(key[i] & 3u));
  w.sp += nc - 1;
  return false;
}

// An any-hit walk's step at inner node w.node of `nodes`: the first hit
// child next, the others pushed.
template <int STACK, bool STATS>
DR_D bool any4_inner(const float4* __restrict__ nodes, const Ray& r, float tmax, Walk4& w, TraceStack<STACK> st,
                     uint32_t* err, TraceStats* stats) {
  int4 ch;
  float ent[4];
  node4_entries_at(nodes, w.node, r, tmax, ent, ch);
  if (STATS) ++stats->nodes;
  int next = kBvh4Empty;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = i4c(ch, k);
    if (!(ent[k] >= 0.0f)) continue;  // a miss, or an empty slot (inverted box)
    if (next == kBvh4Empty) {
      next = c;
    } else if (w.sp < STACK) {
      st.at(w.sp++) = c;
    } else {
      *err |= kErrStackOverflow;
    }
  }
  if (next != kBvh4Empty) {
    w.node = next;
    return false;
  }
  if (w.sp == 0) return true;
  w.node = st.at(--w.sp);
  return false;
}

// One step of a closest-hit walk: an inner node (its hit children, leaves
// and inner nodes alike, are taken nearest first: the nearest now, the
// others pushed far-to-near) or a leaf (its triangles tested against the
// closest hit so far).  Returns true when the walk is over (tbest / best
// then hold the result).
template <int STACK, bool STATS>
DR_D bool closest4_step(const DevScene& S, const Ray& r, int exclude, Walk4& w, float& tbest, int& best,
                        TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  if (--w.budget < 0 || w.node >= S.n_nodes4) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.node < 0) {
    leaf_closest<STATS>(S, w.node, r, exclude, tbest, best, err, stats);
    if (w.sp == 0) return true;
    w.node = st.at(--w.sp);
    return false;
  }
  return closest4_inner<STACK, STATS>(S.nodes4, r, w, tbest, st, err, stats);
}

// One node of an any-hit walk in (tmin, tmax) skipping two triangle ids;
// returns true when the walk is over, with *occluded set.
template <int STACK, bool STATS>
DR_D bool any4_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, Walk4& w, bool* occluded,
                    TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  *occluded = false;
  if (--w.budget < 0 || w.node >= S.n_nodes4) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.node < 0) {
    // a leaf: any hit ends the walk
    if (leaf_any_at<STATS>(S.tris4, S.n_tris, 0, S, w.node, r, tmax, ex0, ex1, err, stats)) {
      *occluded = true;
      return true;
    }
    if (w.sp == 0) return true;
    w.node = st.at(--w.sp);
    return false;
  }
  return any4_inner<STACK, STATS>(S.nodes4, r, tmax, w, st, err, stats);
}

// One step of a 4-wide walk that serves closest-hit rays (any = false) and
// shadow rays (any = true) with the same code, so that a warp holding both
// kinds runs one instruction stream: inner nodes are taken nearest first
// for both (for a shadow ray the order only changes which nodes it visits
// before it finds an occluder, not whether it finds one), and a leaf test
// differs only in what a hit does.  For a closest-hit ray tlim and best are
// the closest hit so far (ex1 is -1); for a shadow ray tlim is its tmax and
// *occluded is set when a triangle other than ex0 and ex1 lies within it.
// The per-triangle tests are those of closest4_step and any4_step, so the
// hits and the occlusion are theirs.  Returns true when the walk is over.
template <int STACK, bool STATS>
DR_D bool mixed4_step(const DevScene& S, const Ray& r, bool any, int ex0, int ex1, Walk4& w, float& tlim, int& best,
                      bool* occluded, TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  if (--w.budget < 0 || w.node >= S.n_nodes4) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.node < 0) {
    const int first = leaf_first(w.node);
    int cnt = leaf_count(w.node);
    if (first + cnt > S.n_tris) {
      *err |= kErrBadIndex;
      cnt = 0;
    }
    for (int i = 0; i < cnt; ++i) {
      const float4 t0 = __ldg(S.tris4 + 3 * (first + i) + 0);
      const float4 t1 = __ldg(S.tris4 + 3 * (first + i) + 1);
      const float4 t2 = __ldg(S.tris4 + 3 * (first + i) + 2);
      const int id = __float_as_int(t0.w);
      if (STATS) ++stats->tris;
      const float tmax = any ? tlim : tlim * 1.0000001f + 1e-30f;
      float th;
      if (id != ex0 && id != ex1 && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tmax, &th)) {
        if (any) {
          *occluded = true;
          return true;
        }
        if (th < tlim || (th == tlim && id < best)) {
          tlim = th;
          best = id;
        }
      }
    }
    if (w.sp == 0) return true;
    w.node = st.at(--w.sp);
    return false;
  }
  return closest4_inner<STACK, STATS>(S.nodes4, r, w, tlim, st, err, stats);
}

template <int STACK, bool STATS>
DR_D int trace_closest4(const DevScene& S, const Ray& r, int exclude, float* t_hit, TraceStack<STACK> st,
                        uint32_t* err, TraceStats* stats) {
  float tbest = __int_as_float(0x7f800000);
  int best = -1;
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    *t_hit = tbest;
    return -1;
  }
  Walk4 w = walk4_begin(S);
  while (!closest4_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats)) {
  }
  *t_hit = tbest;
  return best;
}

template <int STACK, bool STATS>
DR_D bool trace_any4(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, TraceStack<STACK> st,
                     uint32_t* err, TraceStats* stats) {
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    return true;  // treated as occluded
  }
  Walk4 w = walk4_begin(S);
  bool occ = false;
  while (!any4_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, &occ, st, err, stats)) {
  }
  return occ;
}

// Binary-BVH closest hit with t in (tmin, inf), skipping triangle `exclude`
// (original id).  Equal distances resolve to the smaller original triangle
// id.  Returns the original triangle id or -1.
template <int STACK, bool STATS>
DR_D int trace_closest2(const DevScene& S, const Ray& r, int exclude, float* t_hit, TraceStack<STACK> st,
                        uint32_t* err, TraceStats* stats) {
  float tbest = __int_as_float(0x7f800000);
  int best = -1;
  int sp = 0;
  int node = 0;
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    *t_hit = tbest;
    return -1;
  }
  // a tree traversal visits every inner node at most once: more visits mean
  // a corrupt hierarchy, reported instead of looping
  int budget = min(2 * S.n_nodes + 64, kMaxNodeVisits);
  while (true) {
    if (--budget < 0 || node < 0 || node >= S.n_nodes) {
      *err |= kErrBadIndex;
      break;
    }
    float3 lo0, hi0, lo1, hi1;
    int c0, c1;
    load_node(S.nodes, node, lo0, hi0, lo1, hi1, c0, c1);
    if (STATS) ++stats->nodes;
    float e0 = box_entry(lo0, hi0, r, tbest);
    float e1 = box_entry(lo1, hi1, r, tbest);
    // leaves are processed on the spot, inner children are descended into
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = k == 0 ? c0 : c1;
      const float e = k == 0 ? e0 : e1;
      if (c < 0 && e >= 0.0f && e <= tbest) {
        const int first = leaf_first(c);
        int cnt = leaf_count(c);
        if (first + cnt > S.n_tris) {
          *err |= kErrBadIndex;
          cnt = 0;
        }
        for (int i = 0; i < cnt; ++i) {
          const float4 t0 = __ldg(S.tris + 3 * (first + i) + 0);
          const float4 t1 = __ldg(S.tris + 3 * (first + i) + 1);
          const float4 t2 = __ldg(S.tris + 3 * (first + i) + 2);
          const int id = __float_as_int(t0.w);
          if (STATS) ++stats->tris;
          float th;
          if (id != exclude && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tbest * 1.0000001f + 1e-30f, &th)) {
            if (th < tbest || (th == tbest && id < best)) {
              tbest = th;
              best = id;
            }
          }
        }
      }
    }
    const bool in0 = c0 >= 0 && e0 >= 0.0f && e0 <= tbest, in1 = c1 >= 0 && e1 >= 0.0f && e1 <= tbest;
    if (in0 && in1) {
      const int nearc = e0 <= e1 ? c0 : c1, farc = e0 <= e1 ? c1 : c0;
      if (sp < STACK) {
        st.at(sp++) = farc;
      } else {
        *err |= kErrStackOverflow;
      }
      node = nearc;
      continue;
    }
    if (in0) { node = c0; continue; }
    if (in1) { node = c1; continue; }
    // pop, skipping nothing (boxes are re-tested against the shrunken tbest
    // when the popped node's children are examined)
    if (sp == 0) break;
    node = st.at(--sp);
  }
  *t_hit = tbest;
  return best;
}

// Binary-BVH any hit with t in (tmin, tmax), skipping two triangle ids.
template <int STACK, bool STATS>
DR_D bool trace_any2(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, TraceStack<STACK> st,
                     uint32_t* err, TraceStats* stats) {
  int sp = 0;
  int node = 0;
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    return true;  // treated as occluded: no contribution from a broken ray
  }
  int budget = min(2 * S.n_nodes + 64, kMaxNodeVisits);
  while (true) {
    if (--budget < 0 || node < 0 || node >= S.n_nodes) {
      *err |= kErrBadIndex;
      break;
    }
    float3 lo0, hi0, lo1, hi1;
    int c0, c1;
    load_node(S.nodes, node, lo0, hi0, lo1, hi1, c0, c1);
    if (STATS) ++stats->nodes;
    const float e0 = box_entry(lo0, hi0, r, tmax);
    const float e1 = box_entry(lo1, hi1, r, tmax);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = k == 0 ? c0 : c1;
      const float e = k == 0 ? e0 : e1;
      if (c < 0 && e >= 0.0f) {
        const int first = leaf_first(c);
        int cnt = leaf_count(c);
        if (first + cnt > S.n_tris) {
          *err |= kErrBadIndex;
          cnt = 0;
        }
        for (int i = 0; i < cnt; ++i) {
          const float4 t0 = __ldg(S.tris + 3 * (first + i) + 0);
          const float4 t1 = __ldg(S.tris + 3 * (first + i) + 1);
          const float4 t2 = __ldg(S.tris + 3 * (first + i) + 2);
          const int id = __float_as_int(t0.w);
          if (STATS) ++stats->tris;
          float th;
          if (id != ex0 && id != ex1 && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tmax, &th)) return true;
        }
      }
    }
    const bool in0 = c0 >= 0 && e0 >= 0.0f, in1 = c1 >= 0 && e1 >= 0.0f;
    if (in0 && in1) {
      if (sp < STACK) {
        st.at(sp++) = e0 <= e1 ? c1 : c0;
      } else {
        *err |= kErrStackOverflow;
      }
      node = e0 <= e1 ? c0 : c1;
      continue;
    }
    if (in0) { node = c0; continue; }
    if (in1) { node = c1; continue; }
    if (sp == 0) break;
    node = st.at(--sp);
  }
  return false;
}

// ---------------------------------------------------------------- 8-wide
// Compressed 8-wide traversal (node layout at kNode8U4).  A walk holds a
// node group, the hit inner children of one node still to visit (a mask in
// the ray's visit order, slot = position ^ octant), and a triangle group,
// the hit triangles of one node still to test.  A step either tests up to
// four triangles of the triangle group or visits the next child of the node
// group (the rest of the group is pushed first: one stack entry per level).
// Triangles of a node are tested before its children; children come in
// octant order, not sorted by distance.
struct Walk8 {
  uint32_t gbase;  // first inner child of the group's node
  uint32_t gbits;  // bits 0..7: pending children in visit order; bits 8..15: the node's imask
  uint32_t tbase;  // first triangle of the triangle group's node
  uint32_t tbits;  // pending triangles (bit i: triangle tbase + i)
  int sp, budget;
};

DR_D int ray_octant(const Ray& r) {
  return (r.inv.x < 0.0f ? 1 : 0) | (r.inv.y < 0.0f ? 2 : 0) | (r.inv.z < 0.0f ? 4 : 0);
}

// the root as a one-child group (slot 0, an inner child, visit position
// 0 ^ octant); budget: every node once and every triangle step once
DR_D Walk8 walk8_begin(const DevScene& S, const Ray& r) {
  Walk8 w;
  w.gbase = 0;
  w.gbits = (1u << ray_octant(r)) | (1u << 8);
  w.tbase = 0;
  w.tbits = 0;
  w.sp = 0;
  w.budget = min(2 * S.n_nodes8 + S.n_tris / 4 + 64, kMaxNodeVisits);
  return w;
}

DR_D bool walk8_at_tris(const Walk8& w) { return w.tbits != 0u; }

DR_D float byte_f(uint32_t w, int sh) { return (float)((w >> sh) & 0xffu); }

// 2^e for a signed 8-bit exponent in [-100, 100]
DR_D float pow2_of(uint32_t eb, int sh) { return __uint_as_float((uint32_t)((int)(int8_t)(eb >> sh) + 127) << 23); }

// Visits node `node`: tests its eight child boxes against [0, tmax] and
// replaces the walk's groups by the node's hit inner children and hit
// triangles.  Per axis, t = q * (2^e / d) + (p - o) / d: the first product
// is exact (a power of two times 1/d), and the near (far) distances take a
// margin of 2^-21 (|o/d| + |(p - o)/d|) off (on), more than the rounding of
// the two fused multiply-adds, so a box is only ever widened.
DR_D void node8_visit(const DevScene& S, uint32_t node, const Ray& r, float tmax, int oct, Walk8& w) {
  const uint4* nb = S.nodes8 + (size_t)kNode8U4 * node;
  const uint4 h0 = __ldg(nb), h1 = __ldg(nb + 1), qa = __ldg(nb + 2), qb = __ldg(nb + 3), qc = __ldg(nb + 4);
  const float sx = pow2_of(h0.w, 0) * r.inv.x, sy = pow2_of(h0.w, 8) * r.inv.y, sz = pow2_of(h0.w, 16) * r.inv.z;
  const float bx = fmaf(__uint_as_float(h0.x), r.inv.x, -r.oinv.x);
  const float by = fmaf(__uint_as_float(h0.y), r.inv.y, -r.oinv.y);
  const float bz = fmaf(__uint_as_float(h0.z), r.inv.z, -r.oinv.z);
  constexpr float kM = 4.76837158203125e-07f;  // 2^-21
  const float mx = kM * (fabsf(r.oinv.x) + fabsf(bx)), my = kM * (fabsf(r.oinv.y) + fabsf(by)),
              mz = kM * (fabsf(r.oinv.z) + fabsf(bz));
  const float bnx = bx - mx, bfx = bx + mx, bny = by - my, bfy = by + my, bnz = bz - mz, bfz = bz + mz;
  // near planes: lo for a positive direction component, hi for a negative
  const bool nxs = r.inv.x < 0.0f, nys = r.inv.y < 0.0f, nzs = r.inv.z < 0.0f;
  const uint32_t nx0 = nxs ? qb.z : qa.x, nx1 = nxs ? qb.w : qa.y, fx0 = nxs ? qa.x : qb.z, fx1 = nxs ? qa.y : qb.w;
  const uint32_t ny0 = nys ? qc.x : qa.z, ny1 = nys ? qc.y : qa.w, fy0 = nys ? qa.z : qc.x, fy1 = nys ? qa.w : qc.y;
  const uint32_t nz0 = nzs ? qc.z : qb.x, nz1 = nzs ? qc.w : qb.y, fz0 = nzs ? qb.x : qc.z, fz1 = nzs ? qb.y : qc.w;
  uint32_t hits = 0;
#pragma unroll
  for (int sl = 0; sl < 8; ++sl) {
    const int sh = 8 * (sl & 3);
    const float tnx = fmaf(byte_f(sl < 4 ? nx0 : nx1, sh), sx, bnx);
    const float tfx = fmaf(byte_f(sl < 4 ? fx0 : fx1, sh), sx, bfx);
    const float tny = fmaf(byte_f(sl < 4 ? ny0 : ny1, sh), sy, bny);
    const float tfy = fmaf(byte_f(sl < 4 ? fy0 : fy1, sh), sy, bfy);
    const float tnz = fmaf(byte_f(sl < 4 ? nz0 : nz1, sh), sz, bnz);
    const float tfz = fmaf(byte_f(sl < 4 ? fz0 : fz1, sh), sz, bfz);
    const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.0f));
    const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tmax));
    hits |= (tn <= tf * 1.0000002f ? 1u : 0u) << sl;
  }
  const uint32_t im = h0.w >> 24;
  // hit inner children in visit order: slot sl goes to bit sl ^ oct
  uint32_t v = hits & im;
  if (oct & 1) v = ((v & 0x55u) << 1) | ((v >> 1) & 0x55u);
  if (oct & 2) v = ((v & 0x33u) << 2) | ((v >> 2) & 0x33u);
  if (oct & 4) v = ((v & 0x0fu) << 4) | ((v >> 4) & 0x0fu);
  w.gbase = h1.x;
  w.gbits = v | (im << 8);
  // hit leaves: their triangle ranges as one mask
  uint32_t tb = 0;
#pragma unroll
  for (int sl = 0; sl < 8; ++sl) {
    const uint32_t m = ((sl < 4 ? h1.z : h1.w) >> (8 * (sl & 3))) & 0xffu;
    if ((hits >> sl & 1u) && (m & 0x80u)) tb |= ((1u << (((m >> 5) & 3u) + 1u)) - 1u) << (m & 31u);
  }
  w.tbase = h1.y;
  w.tbits = tb;
}

// the next child of the node group: pushes the rest of the group and
// visits the child
template <int STACK>
DR_D void walk8_descend(const DevScene& S, const Ray& r, float tmax, Walk8& w, TraceStack<STACK> st,
                        uint32_t* err) {
  const int oct = ray_octant(r);
  const int k = __ffs(w.gbits & 0xffu) - 1;
  const uint32_t im = w.gbits >> 8;
  const uint32_t node = w.gbase + __popc(im & ((1u << (k ^ oct)) - 1u));
  w.gbits &= ~(1u << k);
  if (w.gbits & 0xffu) {
    if (2 * w.sp + 1 < STACK) {
      st.at(2 * w.sp) = (int)w.gbase;
      st.at(2 * w.sp + 1) = (int)w.gbits;
      ++w.sp;
    } else {
      *err |= kErrStackOverflow;
    }
  }
  if (node >= (uint32_t)S.n_nodes8) {
    *err |= kErrBadIndex;
    w.gbits = 0;
    w.tbits = 0;
    return;
  }
  node8_visit(S, node, r, tmax, oct, w);
}

// after a step: true when the walk is over; else the walk has work
template <int STACK>
DR_D bool walk8_settle(Walk8& w, TraceStack<STACK> st) {
  if (w.tbits != 0u || (w.gbits & 0xffu) != 0u) return false;
  if (w.sp == 0) return true;
  --w.sp;
  w.gbase = (uint32_t)st.at(2 * w.sp);
  w.gbits = (uint32_t)st.at(2 * w.sp + 1);
  return false;
}

template <int STACK, bool STATS>
DR_D bool closest8_step(const DevScene& S, const Ray& r, int exclude, Walk8& w, float& tbest, int& best,
                        TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  if (--w.budget < 0) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.tbits != 0u) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (w.tbits == 0u) break;
      const uint32_t tri = w.tbase + (uint32_t)(__ffs(w.tbits) - 1);
      w.tbits &= w.tbits - 1u;
      if (tri >= (uint32_t)S.n_tris) {
        *err |= kErrBadIndex;
        continue;
      }
      const float4 t0 = __ldg(S.tris8 + 3 * (size_t)tri + 0);
      const float4 t1 = __ldg(S.tris8 + 3 * (size_t)tri + 1);
      const float4 t2 = __ldg(S.tris8 + 3 * (size_t)tri + 2);
      const int id = __float_as_int(t0.w);
      if (STATS) ++stats->tris;
      float th;
      if (id != exclude && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tbest * 1.0000001f + 1e-30f, &th)) {
        if (th < tbest || (th == tbest && id < best)) {
          tbest = th;
          best = id;
        }
      }
    }
  } else {
    walk8_descend<STACK>(S, r, tbest, w, st, err);
    if (STATS) ++stats->nodes;
  }
  return walk8_settle<STACK>(w, st);
}

template <int STACK, bool STATS>
DR_D bool any8_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, Walk8& w, bool* occluded,
                    TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  *occluded = false;
  if (--w.budget < 0) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.tbits != 0u) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (w.tbits == 0u) break;
      const uint32_t tri = w.tbase + (uint32_t)(__ffs(w.tbits) - 1);
      w.tbits &= w.tbits - 1u;
      if (tri >= (uint32_t)S.n_tris) {
        *err |= kErrBadIndex;
        continue;
      }
      const float4 t0 = __ldg(S.tris8 + 3 * (size_t)tri + 0);
      const float4 t1 = __ldg(S.tris8 + 3 * (size_t)tri + 1);
      const float4 t2 = __ldg(S.tris8 + 3 * (size_t)tri + 2);
      const int id = __float_as_int(t0.w);
      if (STATS) ++stats->tris;
      float th;
      if (id != ex0 && id != ex1 && tri_test(xyz(t0), xyz(t1), xyz(t2), r, S.tmin, tmax, &th)) {
        *occluded = true;
        return true;
      }
    }
  } else {
    walk8_descend<STACK>(S, r, tmax, w, st, err);
    if (STATS) ++stats->nodes;
  }
  return walk8_settle<STACK>(w, st);
}

template <int STACK, bool STATS>
DR_D int trace_closest8(const DevScene& S, const Ray& r, int exclude, float* t_hit, TraceStack<STACK> st,
                        uint32_t* err, TraceStats* stats) {
  float tbest = __int_as_float(0x7f800000);
  int best = -1;
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    *t_hit = tbest;
    return -1;
  }
  Walk8 w = walk8_begin(S, r);
  while (!closest8_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats)) {
  }
  *t_hit = tbest;
  return best;
}

template <int STACK, bool STATS>
DR_D bool trace_any8(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, TraceStack<STACK> st,
                     uint32_t* err, TraceStats* stats) {
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    return true;
  }
  Walk8 w = walk8_begin(S, r);
  bool occ = false;
  while (!any8_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, &occ, st, err, stats)) {
  }
  return occ;
}

// ---------------------------------------------------------------- two-level
// Walk of a two-level BVH (instanced scenes): the 4-wide walk over the TLAS
// in world space; a TLAS leaf (one instance) maps the ray into the
// instance's object space (the parameter t is unchanged by the affine map),
// pushes a return mark (kBvh4Empty) and continues at the instance's BLAS
// root; popping the mark returns to the TLAS.  Hits are global triangle ids
// (the instance's first id + the id within its mesh).
struct WalkTL {
  Walk4 w;    // node: a TLAS node at the top level, else a BLAS node
  int inst;   // current instance; -1 at the top level
  int tbase;  // global id of the instance's first triangle
  Ray ro;     // the ray in the instance's object space
};

DR_D WalkTL walktl_begin(const DevScene&) {
  WalkTL w;
  w.w = Walk4{0, 0, kMaxNodeVisits};
  w.inst = -1;
  w.tbase = 0;
  return w;
}

DR_D bool walktl_at_leaf(const WalkTL& w) { return w.w.node < 0; }

// Enters instance `inst` from a TLAS leaf: object-space ray, return mark,
// BLAS root.  Returns false on a bad record (the walk then ends).
template <int STACK>
DR_D bool walktl_enter(const DevScene& S, const Ray& r, WalkTL& w, TraceStack<STACK> st, uint32_t* err) {
  const int inst = leaf_first(w.w.node);
  if (inst >= S.n_insts) {
    *err |= kErrBadIndex;
    return false;
  }
  const float4* ir = S.insts + (size_t)kInstF4 * inst;
  const float4 m0 = __ldg(ir), m1 = __ldg(ir + 1), m2 = __ldg(ir + 2);
  const int4 i3 = __ldg(reinterpret_cast<const int4*>(ir + 3));
  const float3 o = f3(fmaf(m0.x, r.o.x, fmaf(m0.y, r.o.y, fmaf(m0.z, r.o.z, m0.w))),
                      fmaf(m1.x, r.o.x, fmaf(m1.y, r.o.y, fmaf(m1.z, r.o.z, m1.w))),
                      fmaf(m2.x, r.o.x, fmaf(m2.y, r.o.y, fmaf(m2.z, r.o.z, m2.w))));
  const float3 d = f3(fmaf(m0.x, r.d.x, fmaf(m0.y, r.d.y, m0.z * r.d.z)),
                      fmaf(m1.x, r.d.x, fmaf(m1.y, r.d.y, m1.z * r.d.z)),
                      fmaf(m2.x, r.d.x, fmaf(m2.y, r.d.y, m2.z * r.d.z)));
  w.ro = make_ray(o, d);
  w.inst = inst;
  w.tbase = i3.y;
  if (w.w.sp < STACK) {
    st.at(w.w.sp++) = kBvh4Empty;
  } else {
    *err |= kErrStackOverflow;
    return false;
  }
  w.w.node = i3.x;
  return true;
}

// pops the next entry (a return mark switches back to the TLAS); true when
// the walk is over
template <int STACK>
DR_D bool walktl_pop(WalkTL& w, TraceStack<STACK> st) {
  while (true) {
    if (w.w.sp == 0) return true;
    w.w.node = st.at(--w.w.sp);
    if (w.w.node != kBvh4Empty) return false;
    w.inst = -1;
  }
}

template <int STACK, bool STATS>
DR_D bool closest_tl_step(const DevScene& S, const Ray& r, int exclude, WalkTL& w, float& tbest, int& best,
                          TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  const bool top = w.inst < 0;
  if (--w.w.budget < 0 || w.w.node >= (top ? S.n_tl_nodes : S.n_bl_nodes)) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.w.node < 0) {
    if (top) return walktl_enter<STACK>(S, r, w, st, err) ? false : true;
    leaf_closest_at<STATS>(S.bl_tris, S.n_bl_tris, w.tbase, S, w.w.node, w.ro, exclude, tbest, best, err, stats);
    return walktl_pop<STACK>(w, st);
  }
  const int sp0 = w.w.sp;
  const bool done = closest4_inner<STACK, STATS>(top ? S.tl_nodes : S.bl_nodes, top ? r : w.ro, w.w, tbest, st, err,
                                                 stats);
  // a pop inside the inner step may have taken a return mark
  if (!done && w.w.sp < sp0 && w.w.node == kBvh4Empty) {
    w.inst = -1;
    return walktl_pop<STACK>(w, st);
  }
  return done;
}

template <int STACK, bool STATS>
DR_D bool any_tl_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, WalkTL& w, bool* occluded,
                      TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  *occluded = false;
  const bool top = w.inst < 0;
  if (--w.w.budget < 0 || w.w.node >= (top ? S.n_tl_nodes : S.n_bl_nodes)) {
    *err |= kErrBadIndex;
    return true;
  }
  if (w.w.node < 0) {
    if (top) return walktl_enter<STACK>(S, r, w, st, err) ? false : true;
    if (leaf_any_at<STATS>(S.bl_tris, S.n_bl_tris, w.tbase, S, w.w.node, w.ro, tmax, ex0, ex1, err, stats)) {
      *occluded = true;
      return true;
    }
    return walktl_pop<STACK>(w, st);
  }
  const int sp0 = w.w.sp;
  const bool done = any4_inner<STACK, STATS>(top ? S.tl_nodes : S.bl_nodes, top ? r : w.ro, tmax, w.w, st, err, stats);
  if (!done && w.w.sp < sp0 && w.w.node == kBvh4Empty) {
    w.inst = -1;
    return walktl_pop<STACK>(w, st);
  }
  return done;
}

template <int STACK, bool STATS>
DR_D int trace_closest_tl(const DevScene& S, const Ray& r, int exclude, float* t_hit, TraceStack<STACK> st,
                          uint32_t* err, TraceStats* stats) {
  float tbest = __int_as_float(0x7f800000);
  int best = -1;
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    *t_hit = tbest;
    return -1;
  }
  WalkTL w = walktl_begin(S);
  while (!closest_tl_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats)) {
  }
  *t_hit = tbest;
  return best;
}

template <int STACK, bool STATS>
DR_D bool trace_any_tl(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, TraceStack<STACK> st,
                       uint32_t* err, TraceStats* stats) {
  if (!ray_finite(r.o, r.d)) {
    *err |= kErrNonFinite;
    return true;
  }
  WalkTL w = walktl_begin(S);
  bool occ = false;
  while (!any_tl_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, &occ, st, err, stats)) {
  }
  return occ;
}

// Width-generic walk interface of the persistent passes.
template <int WIDTH>
struct WalkOf {
  using type = Walk4;
};
template <>
struct WalkOf<8> {
  using type = Walk8;
};
constexpr int kWalkTwoLevel = 1;  // the WIDTH of the two-level walk
template <>
struct WalkOf<kWalkTwoLevel> {
  using type = WalkTL;
};
DR_D void walk_begin(const DevScene& S, const Ray&, Walk4& w) { w = walk4_begin(S); }
DR_D void walk_begin(const DevScene& S, const Ray& r, Walk8& w) { w = walk8_begin(S, r); }
DR_D bool walk_at_leaf(const Walk4& w) { return w.node < 0; }
DR_D bool walk_at_leaf(const Walk8& w) { return w.tbits != 0u; }
DR_D void walk_begin(const DevScene& S, const Ray&, WalkTL& w) { w = walktl_begin(S); }
DR_D bool walk_at_leaf(const WalkTL& w) { return walktl_at_leaf(w); }
template <int STACK, bool STATS>
DR_D bool closest_step(const DevScene& S, const Ray& r, int exclude, WalkTL& w, float& tbest, int& best,
                       TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return closest_tl_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats);
}
template <int STACK, bool STATS>
DR_D bool any_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, WalkTL& w, bool* occluded,
                   TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return any_tl_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, occluded, st, err, stats);
}
template <int STACK, bool STATS>
DR_D bool closest_step(const DevScene& S, const Ray& r, int exclude, Walk4& w, float& tbest, int& best,
                       TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return closest4_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats);
}
template <int STACK, bool STATS>
DR_D bool closest_step(const DevScene& S, const Ray& r, int exclude, Walk8& w, float& tbest, int& best,
                       TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return closest8_step<STACK, STATS>(S, r, exclude, w, tbest, best, st, err, stats);
}
template <int STACK, bool STATS>
DR_D bool any_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, Walk4& w, bool* occluded,
                   TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return any4_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, occluded, st, err, stats);
}
template <int STACK, bool STATS>
DR_D bool any_step(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, Walk8& w, bool* occluded,
                   TraceStack<STACK> st, uint32_t* err, TraceStats* stats) {
  return any8_step<STACK, STATS>(S, r, tmax, ex0, ex1, w, occluded, st, err, stats);
}

// Closest hit / any hit through whichever BVH the scene selects (WIDTH 0:
// decided per call from S.nodes4; 2, 4 or 8: fixed at compile time, for
// kernels specialised per width).
template <int STACK, bool STATS, int WIDTH = 0>
DR_D int trace_closest(const DevScene& S, const Ray& r, int exclude, float* t_hit, TraceStack<STACK> st,
                       uint32_t* err, TraceStats* stats) {
  if (WIDTH == 8) return trace_closest8<STACK, STATS>(S, r, exclude, t_hit, st, err, stats);
  if (WIDTH == kWalkTwoLevel) return trace_closest_tl<STACK, STATS>(S, r, exclude, t_hit, st, err, stats);
  if (WIDTH == 4 || (WIDTH == 0 && S.nodes4 != nullptr))
    return trace_closest4<STACK, STATS>(S, r, exclude, t_hit, st, err, stats);
  return trace_closest2<STACK, STATS>(S, r, exclude, t_hit, st, err, stats);
}

template <int STACK, bool STATS, int WIDTH = 0>
DR_D bool trace_any(const DevScene& S, const Ray& r, float tmax, int ex0, int ex1, TraceStack<STACK> st,
                    uint32_t* err, TraceStats* stats) {
  if (WIDTH == 8) return trace_any8<STACK, STATS>(S, r, tmax, ex0, ex1, st, err, stats);
  if (WIDTH == kWalkTwoLevel) return trace_any_tl<STACK, STATS>(S, r, tmax, ex0, ex1, st, err, stats);
  if (WIDTH == 4 || (WIDTH == 0 && S.nodes4 != nullptr))
    return trace_any4<STACK, STATS>(S, r, tmax, ex0, ex1, st, err, stats);
  return trace_any2<STACK, STATS>(S, r, tmax, ex0, ex1, st, err, stats);
}

}  // namespace dr
