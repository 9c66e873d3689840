// Collapse of the binary BVH into a 4-wide BVH, on the device, at scene
// upload.
//
// The 4-wide tree is the one of least surface-area-heuristic cost (unit
// cost per node visit and per triangle test, weighted by box area) that
// regroups the binary tree's nodes, found by dynamic programming over the
// binary tree: for every binary node n and k = 1..4 the cheapest way to
// place n's subtree into at most k child slots of a 4-wide node (one slot:
// n as a leaf of at most kBvh4MaxLeaf triangles, or as a 4-wide node of its
// own; more slots: n's two children share them).  The 8-wide collapse
// widens greedily: starting from a binary node's two children, the inner
// child of largest surface area is replaced by its own two children until
// there are eight children or only leaves are left.
// Triangles are re-laid in the binary tree's depth-first order, so every
// subtree (hence every 4-wide leaf) is one contiguous range.
//
// Passes (deterministic: no result depends on thread arrival order):
//   parents      parent index of every inner node, and reference counts
//                of every inner node and triangle (the tree check: each
//                inner node but the root, and each triangle, referenced
//                exactly once)
//   bottom-up    triangle count and SAH cost per node (the thread that
//                delivers a node's second finished child settles it; no
//                thread ever waits for another)
//   first        depth-first position of every subtree's first triangle,
//                and every inner node's depth (the binary tree's height)
//   mark         top-down, one launch per 4-wide level: which binary nodes
//                become 4-wide nodes, their depth and stack need
//   scan         4-wide node slots in binary-node order
//   emit         the 4-wide nodes and the re-laid triangles
//
// The 8-wide compressed collapse shares the first four passes and the leaf
// decision, then numbers its nodes breadth first so that each node's inner
// children are consecutive (per level: count, scan, place), lays out each
// node's leaf triangles consecutively, and emits quantised nodes.
#include <algorithm>
#include <cmath>

#include "dr_internal.h"

namespace dr {

namespace {

constexpr int kB4Threads = 256;

struct Kid {
  int code;    // binary child link: >= 0 inner node, < 0 binary leaf
  int parent;  // binary node holding the link
  int side;    // 0 / 1: which of the parent's two links
  float3 lo, hi;
};

DR_D Kid kid_of(const float4* __restrict__ n2, int node, int k) {
  const float4 a = n2[4 * node + 0], b = n2[4 * node + 1], c = n2[4 * node + 2], d = n2[4 * node + 3];
  Kid r;
  r.code = __float_as_int(k == 0 ? d.x : d.y);
  r.parent = node;
  r.side = k;
  if (k == 0) {
    r.lo = f3(a.x, a.y, a.z);
    r.hi = f3(a.w, b.x, b.y);
  } else {
    r.lo = f3(b.z, b.w, c.x);
    r.hi = f3(c.y, c.z, c.w);
  }
  return r;
}

DR_D float box_area(float3 lo, float3 hi) {
  const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
  return (dx < 0.0f || dy < 0.0f || dz < 0.0f) ? 0.0f : 2.0f * (dx * dy + dy * dz + dz * dx);
}

struct B4Scratch {
  int* parent;        // [nn] (-1 at the root)
  int* cnt;           // [nn] triangles below
  float* cost;        // [nn] SAH cost of the subtree
  uint32_t* visit;    // [nn] bottom-up arrivals
  int* first;         // [nn] depth-first position of the first triangle
  uint32_t* is4;      // [nn] 1: becomes a 4-wide inner node
  uint32_t* slot;     // [nn] exclusive scan of is4
  int* need;          // [nn] stack entries held by the ancestors
  int* depth;         // [nn] 4-wide depth (root = 1)
  uint32_t* queue[2]; // [nn] each
  uint8_t* as_leaf;   // [nn] 1: becomes one 4-wide leaf
  uint32_t* refs;     // [nn] references to each inner node
  uint32_t* tri_refs; // [nt] references to each triangle
  uint32_t* counts;   // [8]: queue sizes (2), max need, max 4-wide depth, max binary depth
  uint32_t* err;      // [1]
  float* dp_cost;     // [nn][4]: [0] the subtree in one slot, [k - 1] in k = 2..4 slots shared by its children
  uint8_t* dp_split;  // [nn][4]: [k - 1] slots of the left child when k = 2..4 slots are shared
  void* scan_tmp;
};

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

size_t b4_bytes(int nn, int nt) {
  const size_t n = (size_t)nn;
  return a256(n * 4) * 12 + a256((size_t)nt * 4) + a256(n) + a256(32) + a256(4) + a256(n * 16) + a256(n * 4) +
         a256(scan_scratch_bytes(n));
}

B4Scratch b4_carve(void* base, int nn, int nt) {
  const size_t n = (size_t)nn;
  char* p = static_cast<char*>(base);
  B4Scratch s;
  s.parent = reinterpret_cast<int*>(p); p += a256(n * 4);
  s.cnt = reinterpret_cast<int*>(p); p += a256(n * 4);
  s.cost = reinterpret_cast<float*>(p); p += a256(n * 4);
  s.visit = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.first = reinterpret_cast<int*>(p); p += a256(n * 4);
  s.is4 = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.slot = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.need = reinterpret_cast<int*>(p); p += a256(n * 4);
  s.depth = reinterpret_cast<int*>(p); p += a256(n * 4);
  s.queue[0] = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.queue[1] = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.refs = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  s.tri_refs = reinterpret_cast<uint32_t*>(p); p += a256((size_t)nt * 4);
  s.as_leaf = reinterpret_cast<uint8_t*>(p); p += a256(n);
  s.counts = reinterpret_cast<uint32_t*>(p); p += a256(32);
  s.err = reinterpret_cast<uint32_t*>(p); p += a256(4);
  s.dp_cost = reinterpret_cast<float*>(p); p += a256(n * 16);
  s.dp_split = reinterpret_cast<uint8_t*>(p); p += a256(n * 4);
  s.scan_tmp = p;
  return s;
}

// triangles below a binary link
DR_D int count_of(int code, const int* cnt) { return code < 0 ? leaf_count(code) : cnt[code]; }

__global__ void parents_kernel(const float4* __restrict__ n2, int nn, int nt, int* parent, uint32_t* visit,
                               uint32_t* is4, int* need, int* depth, uint32_t* refs, uint32_t* tri_refs,
                               uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  visit[n] = 0;
  is4[n] = n == 0 ? 1u : 0u;
  if (n == 0) {
    need[0] = 0;
    depth[0] = 1;
  }
  const float4 d = n2[4 * n + 3];
  const int c[2] = {__float_as_int(d.x), __float_as_int(d.y)};
  for (int k = 0; k < 2; ++k) {
    if (c[k] >= 0) {
      if (c[k] == 0 || c[k] >= nn) {
        atomicOr(err, kErrBadIndex);
      } else {
        parent[c[k]] = n;
        atomicAdd(&refs[c[k]], 1u);
      }
    } else {
      const int first = leaf_first(c[k]), cnt = leaf_count(c[k]);
      if (first + cnt > nt) atomicOr(err, kErrBadIndex);
      else
        for (int i = 0; i < cnt; ++i) atomicAdd(&tri_refs[first + i], 1u);
    }
  }
}

// the tree check: the root unreferenced, every other inner node and every
// triangle referenced exactly once
__global__ void verify_kernel(int nn, int nt, const uint32_t* refs, const uint32_t* tri_refs, uint32_t* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn && refs[i] != (i == 0 ? 0u : 1u)) atomicOr(err, kErrBadIndex);
  if (i < nt && tri_refs[i] != 1u) atomicOr(err, kErrBadIndex);
}

// Area-weighted SAH cost of placing child reference c into at most k slots
// (a binary leaf link takes one slot as it is).
DR_D float slots_cost(const Kid& c, int k, const float* dp_cost) {
  if (c.code < 0) return box_area(c.lo, c.hi) * (float)leaf_count(c.code);
  const volatile float* d = dp_cost + 4 * (size_t)c.code;
  float best = d[0];
  for (int i = 2; i <= k; ++i) best = fminf(best, d[i - 1]);
  return best;
}

// settles node n (its inner children are settled): count, binary SAH cost,
// and the collapse's dynamic programme (see the file comment): the costs of
// n's subtree in one slot and in 2..4 slots shared by its children, the
// best split of those slots, and whether n in one slot is a leaf
DR_D void settle(const float4* __restrict__ n2, int n, int* cnt, float* cost, uint8_t* as_leaf, float* dp_cost,
                 uint8_t* dp_split, int max_leaf) {
  const Kid k0 = kid_of(n2, n, 0), k1 = kid_of(n2, n, 1);
  const float an_raw = box_area(f3(fminf(k0.lo.x, k1.lo.x), fminf(k0.lo.y, k1.lo.y), fminf(k0.lo.z, k1.lo.z)),
                                f3(fmaxf(k0.hi.x, k1.hi.x), fmaxf(k0.hi.y, k1.hi.y), fmaxf(k0.hi.z, k1.hi.z)));
  const float an = fmaxf(an_raw, 1e-30f);
  int total = 0;
  float c_inner = 1.0f;
  for (int k = 0; k < 2; ++k) {
    const Kid& c = k == 0 ? k0 : k1;
    int cc;
    float ccost;
    if (c.code < 0) {
      cc = leaf_count(c.code);
      ccost = (float)cc;
    } else {
      cc = *(volatile const int*)(cnt + c.code);
      ccost = *(volatile const float*)(cost + c.code);
    }
    total += cc;
    c_inner += box_area(c.lo, c.hi) / an * ccost;
  }
  float* dc = dp_cost + 4 * (size_t)n;
  uint8_t* ds = dp_split + 4 * (size_t)n;
  for (int k = 2; k <= 4; ++k) {
    float best = 3.0e38f;
    int bj = 1;
    for (int j = 1; j < k; ++j) {
      const float c = slots_cost(k0, j, dp_cost) + slots_cost(k1, k - j, dp_cost);
      if (c < best) {
        best = c;
        bj = j;
      }
    }
    dc[k - 1] = best;
    ds[k - 1] = (uint8_t)bj;
  }
  const float node_cost = an_raw + dc[3];
  const bool leaf = total <= max_leaf && an_raw * (float)total <= node_cost;
  dc[0] = leaf ? an_raw * (float)total : node_cost;
  ds[0] = 0;
  cnt[n] = total;
  cost[n] = leaf ? (float)total : c_inner;
  as_leaf[n] = leaf ? 1 : 0;
}

// Each node with leaf links starts a walk towards the root; a node is
// settled by the walk that brings its second finished child, the first
// arrival ends its walk there.
__global__ void bottom_up_kernel(const float4* __restrict__ n2, int nn, const int* parent, int* cnt, float* cost,
                                 uint8_t* as_leaf, float* dp_cost, uint8_t* dp_split, uint32_t* visit, int max_leaf,
                                 uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const float4 d = n2[4 * n + 3];
  const uint32_t leaves = (__float_as_int(d.x) < 0 ? 1u : 0u) + (__float_as_int(d.y) < 0 ? 1u : 0u);
  if (leaves == 0) return;
  if (atomicAdd(&visit[n], leaves) + leaves < 2) return;
  __threadfence();
  int cur = n;
  for (int guard = 0; guard <= nn; ++guard) {
    settle(n2, cur, cnt, cost, as_leaf, dp_cost, dp_split, max_leaf);
    const int p = parent[cur];
    if (p < 0) return;
    __threadfence();  // cur's results visible before its arrival is counted
    if (atomicAdd(&visit[p], 1u) == 0) return;
    __threadfence();
    cur = p;
  }
  atomicOr(err, kErrBadIndex);
}

// depth-first position of node n's first triangle: the triangles below
// every left sibling on the way up come before it
__global__ void first_kernel(const float4* __restrict__ n2, int nn, const int* parent, const int* cnt, int* first,
                             uint32_t* max_depth, uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  int f = 0, cur = n;
  for (int guard = 0; guard <= nn; ++guard) {
    const int p = parent[cur];
    if (p < 0) {
      first[n] = f;
      atomicMax(max_depth, (uint32_t)guard + 1u);
      return;
    }
    const float4 d = n2[4 * p + 3];
    if (__float_as_int(d.y) == cur) f += count_of(__float_as_int(d.x), cnt);
    cur = p;
  }
  atomicOr(err, kErrBadIndex);
}

DR_D bool leaf_ref(const Kid& k, const uint8_t* as_leaf) { return k.code < 0 || as_leaf[k.code]; }

// greedy widening of binary node n to up to W children
template <int W = 4>
DR_D int expand(const float4* __restrict__ n2, int n, const uint8_t* as_leaf, Kid kids[W]) {
  kids[0] = kid_of(n2, n, 0);
  kids[1] = kid_of(n2, n, 1);
  int nk = 2;
  while (nk < W) {
    int best = -1;
    float ba = -1.0f;
    for (int i = 0; i < nk; ++i) {
      if (leaf_ref(kids[i], as_leaf)) continue;
      const float a = box_area(kids[i].lo, kids[i].hi);
      if (a > ba) {
        ba = a;
        best = i;
      }
    }
    if (best < 0) break;
    const int id = kids[best].code;
    for (int i = best; i + 1 < nk; ++i) kids[i] = kids[i + 1];
    kids[nk - 1] = kid_of(n2, id, 0);
    kids[nk] = kid_of(n2, id, 1);
    ++nk;
  }
  return nk;
}

// The children of 4-wide node n: the binary subtree distributed over four
// slots by the dynamic programme's choices (a reference that is best in one
// slot becomes a child, else its two children share its slots).
DR_D int expand_dp(const float4* __restrict__ n2, int n, const float* dp_cost, const uint8_t* dp_split,
                   Kid kids[4]) {
  struct Item {
    Kid c;
    int k;
  };
  Item st[4];
  int sp = 0, nk = 0;
  const int j = dp_split[4 * (size_t)n + 3];
  st[sp++] = Item{kid_of(n2, n, 1), 4 - j};
  st[sp++] = Item{kid_of(n2, n, 0), j};
  while (sp > 0 && nk < 4) {
    const Item it = st[--sp];
    const Kid& c = it.c;
    int bk = 1;
    if (c.code >= 0) {
      const float* d = dp_cost + 4 * (size_t)c.code;
      float best = d[0];
      for (int i = 2; i <= it.k; ++i)
        if (d[i - 1] < best) {
          best = d[i - 1];
          bk = i;
        }
    }
    if (bk == 1 || sp + 2 > 4) {
      kids[nk++] = c;
    } else {
      const int jj = dp_split[4 * (size_t)c.code + bk - 1];
      st[sp++] = Item{kid_of(n2, c.code, 1), bk - jj};
      st[sp++] = Item{kid_of(n2, c.code, 0), jj};
    }
  }
  return nk;
}

__global__ void mark_kernel(const float4* __restrict__ n2, const uint8_t* as_leaf, const float* dp_cost,
                            const uint8_t* dp_split, const uint32_t* q_in, uint32_t n_in, uint32_t* q_out,
                            uint32_t* n_out, uint32_t* is4, int* need, int* depth, uint32_t* maxes) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_in) return;
  const int n = (int)q_in[t];
  Kid kids[4];
  const int nk = expand_dp(n2, n, dp_cost, dp_split, kids);
  // a closest-hit walk pushes every hit child but the nearest (leaves too)
  const int here = need[n] + max(0, nk - 1);
  atomicMax(&maxes[0], (uint32_t)here);
  atomicMax(&maxes[1], (uint32_t)depth[n]);
  for (int k = 0; k < nk; ++k) {
    if (leaf_ref(kids[k], as_leaf)) continue;
    const int c = kids[k].code;
    is4[c] = 1;
    need[c] = here;
    depth[c] = depth[n] + 1;
    q_out[atomicAdd(n_out, 1u)] = (uint32_t)c;
  }
}

// copies the triangles of binary node n's leaf links to their depth-first
// place in t4
DR_D void relayout_links(const float4* __restrict__ n2, const float4* __restrict__ t2, int n, int nt, const int* cnt,
                         const int* first, float4* __restrict__ t4, uint32_t* err) {
  const float4 dn = n2[4 * n + 3];
  for (int k = 0; k < 2; ++k) {
    const int code = __float_as_int(k == 0 ? dn.x : dn.y);
    if (code >= 0) continue;
    const int pos = first[n] + (k == 1 ? count_of(__float_as_int(dn.x), cnt) : 0);
    const int src = leaf_first(code), m = leaf_count(code);
    if (pos < 0 || pos + m > nt || src + m > nt) {
      atomicOr(err, kErrBadIndex);
      continue;
    }
    for (int i = 0; i < m; ++i)
      for (int q = 0; q < kTriF4; ++q) t4[(size_t)kTriF4 * (pos + i) + q] = t2[(size_t)kTriF4 * (src + i) + q];
  }
}

// depth-first position and count of the triangles of a leaf reference
DR_D void leaf_range(const float4* __restrict__ n2, const Kid& c, const int* cnt, const int* first, int* pos,
                     int* count) {
  if (c.code >= 0) {
    *pos = first[c.code];
    *count = cnt[c.code];
  } else {
    const float4 d = n2[4 * c.parent + 3];
    *pos = first[c.parent] + (c.side == 1 ? count_of(__float_as_int(d.x), cnt) : 0);
    *count = leaf_count(c.code);
  }
}

__global__ void emit_kernel(const float4* __restrict__ n2, const float4* __restrict__ t2, int nn, int nt,
                            const uint8_t* as_leaf, const float* dp_cost, const uint8_t* dp_split, const int* cnt,
                            const int* first, const uint32_t* is4, const uint32_t* slot, float4* __restrict__ n4,
                            float4* __restrict__ t4, uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  // triangles of this node's binary leaf links, to their depth-first place
  relayout_links(n2, t2, n, nt, cnt, first, t4, err);
  if (!is4[n]) return;
  Kid kids[4];
  const int nk = expand_dp(n2, n, dp_cost, dp_split, kids);
  // an empty slot holds an inverted box (lo = +inf, hi = -inf), which every
  // slab test misses, so the walk needs no test of its link
  float lo[3][4], hi[3][4];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 4; ++k) {
      lo[a][k] = __int_as_float(0x7f800000);
      hi[a][k] = __int_as_float(0xff800000);
    }
  int links[4] = {kBvh4Empty, kBvh4Empty, kBvh4Empty, kBvh4Empty};
  for (int k = 0; k < nk; ++k) {
    const Kid& c = kids[k];
    lo[0][k] = c.lo.x; lo[1][k] = c.lo.y; lo[2][k] = c.lo.z;
    hi[0][k] = c.hi.x; hi[1][k] = c.hi.y; hi[2][k] = c.hi.z;
    if (!leaf_ref(c, as_leaf)) {
      links[k] = (int)slot[c.code];
    } else {
      int pos, m;
      leaf_range(n2, c, cnt, first, &pos, &m);
      links[k] = leaf_code(pos, m);
    }
  }
  float4* o = n4 + (size_t)kNode4F4 * slot[n];
  o[0] = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
  o[1] = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
  o[2] = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
  o[3] = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
  o[4] = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
  o[5] = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
  o[6] = make_float4(__int_as_float(links[0]), __int_as_float(links[1]), __int_as_float(links[2]),
                     __int_as_float(links[3]));
}

// ---------------------------------------------------------------- 8-wide
// Slots of up to eight children by the octant heuristic: slot s is visited
// first by rays of octant s, so it goes to the child nearest along that
// octant's diagonal direction (smallest projection of its centre offset);
// pairs are assigned greedily, globally smallest projection first.
DR_D void assign_slots(const Kid* kids, int nk, int slot_of[8]) {
  float3 lo = kids[0].lo, hi = kids[0].hi;
  for (int k = 1; k < nk; ++k) {
    lo = f3(fminf(lo.x, kids[k].lo.x), fminf(lo.y, kids[k].lo.y), fminf(lo.z, kids[k].lo.z));
    hi = f3(fmaxf(hi.x, kids[k].hi.x), fmaxf(hi.y, kids[k].hi.y), fmaxf(hi.z, kids[k].hi.z));
  }
  const float3 c = (lo + hi) * 0.5f;
  uint32_t used_k = 0, used_s = 0;
  for (int round = 0; round < nk; ++round) {
    float best = INFINITY;
    int bk = -1, bs = -1;
    for (int k = 0; k < nk; ++k) {
      if (used_k >> k & 1u) continue;
      const float3 v = (kids[k].lo + kids[k].hi) * 0.5f - c;
      for (int sl = 0; sl < 8; ++sl) {
        if (used_s >> sl & 1u) continue;
        const float cost = (sl & 1 ? -v.x : v.x) + (sl & 2 ? -v.y : v.y) + (sl & 4 ? -v.z : v.z);
        if (bk < 0 || cost < best) {
          best = cost;
          bk = k;
          bs = sl;
        }
      }
    }
    slot_of[bk] = bs;
    used_k |= 1u << bk;
    used_s |= 1u << bs;
  }
}

// child index per slot (-1: empty)
DR_D void kids_by_slot(const Kid* kids, int nk, int by_slot[8]) {
  int slot_of[8];
  assign_slots(kids, nk, slot_of);
  for (int sl = 0; sl < 8; ++sl) by_slot[sl] = -1;
  for (int k = 0; k < nk; ++k) by_slot[slot_of[k]] = k;
}

// level pass 1: inner children and leaf triangles of each node of the level
__global__ void count8_kernel(const float4* __restrict__ n2, const uint8_t* as_leaf, const int* cnt, const int* first,
                              const uint32_t* q_in, uint32_t n_in, uint32_t base_cur, uint32_t* n_inner,
                              uint32_t* tri_cnt, uint32_t* err) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_in) return;
  Kid kids[8];
  const int nk = expand<8>(n2, (int)q_in[i], as_leaf, kids);
  uint32_t inner = 0, tris = 0;
  for (int k = 0; k < nk; ++k) {
    if (!leaf_ref(kids[k], as_leaf)) {
      ++inner;
    } else {
      int pos, m;
      leaf_range(n2, kids[k], cnt, first, &pos, &m);
      if (m < 1 || m > kBvh4MaxLeaf) atomicOr(err, kErrBadIndex);
      tris += (uint32_t)m;
    }
  }
  n_inner[i] = inner;
  tri_cnt[base_cur + i] = tris;
}

// level pass 2: node numbers (breadth first; a node's inner children
// consecutive, in slot order) and the next level's queue
__global__ void place8_kernel(const float4* __restrict__ n2, const uint8_t* as_leaf, const uint32_t* q_in,
                              uint32_t n_in, const uint32_t* pos, uint32_t base_cur, uint32_t base_next,
                              uint32_t* q_out, uint32_t* bfs, uint32_t* child_base) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_in) return;
  const int n = (int)q_in[i];
  bfs[base_cur + i] = (uint32_t)n;
  child_base[base_cur + i] = base_next + pos[i];
  Kid kids[8];
  const int nk = expand<8>(n2, n, as_leaf, kids);
  int by_slot[8];
  kids_by_slot(kids, nk, by_slot);
  uint32_t r = 0;
  for (int sl = 0; sl < 8; ++sl) {
    const int k = by_slot[sl];
    if (k >= 0 && !leaf_ref(kids[k], as_leaf)) q_out[pos[i] + r++] = (uint32_t)kids[k].code;
  }
}

__global__ void relayout_kernel(const float4* __restrict__ n2, const float4* __restrict__ t2, int nn, int nt,
                                const int* cnt, const int* first, float4* __restrict__ tdfs, uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nn) relayout_links(n2, t2, n, nt, cnt, first, tdfs, err);
}

// quantisation of one axis: exponent e with 255 * 2^e >= hi - lo, and the
// conservative 8-bit planes of each child (computed in FP64, exact)
DR_D int axis_exponent(float lo, float hi) {
  const double ext = (double)hi - (double)lo;
  int e = ext > 0.0 ? (int)ceil(log2(ext / 255.0)) : -100;
  e = max(-100, min(100, e));
  while (e < 100 && ldexp(255.0, e) < ext) ++e;
  return e;
}
DR_D uint32_t q_lo(float p, int e, float v) {
  const double sc = ldexp(1.0, e);
  double q = floor(((double)v - (double)p) / sc);
  q = fmin(fmax(q, 0.0), 255.0);
  while (q > 0.0 && (double)p + q * sc > (double)v) q -= 1.0;
  return (uint32_t)q;
}
DR_D uint32_t q_hi(float p, int e, float v) {
  const double sc = ldexp(1.0, e);
  double q = ceil(((double)v - (double)p) / sc);
  q = fmin(fmax(q, 0.0), 255.0);
  return (uint32_t)q;
}

__global__ void emit8_kernel(const float4* __restrict__ n2, uint32_t n_wide, const uint8_t* as_leaf, const int* cnt,
                             const int* first, const uint32_t* bfs, const uint32_t* child_base,
                             const uint32_t* tri_base, const float4* __restrict__ tdfs, int nt,
                             uint4* __restrict__ n8, float4* __restrict__ t8, uint32_t* err) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_wide) return;
  Kid kids[8];
  const int nk = expand<8>(n2, (int)bfs[i], as_leaf, kids);
  int by_slot[8];
  kids_by_slot(kids, nk, by_slot);
  float3 lo = kids[0].lo, hi = kids[0].hi;
  for (int k = 1; k < nk; ++k) {
    lo = f3(fminf(lo.x, kids[k].lo.x), fminf(lo.y, kids[k].lo.y), fminf(lo.z, kids[k].lo.z));
    hi = f3(fmaxf(hi.x, kids[k].hi.x), fmaxf(hi.y, kids[k].hi.y), fmaxf(hi.z, kids[k].hi.z));
  }
  const int ex = axis_exponent(lo.x, hi.x), ey = axis_exponent(lo.y, hi.y), ez = axis_exponent(lo.z, hi.z);
  uint32_t qlx[2] = {0, 0}, qly[2] = {0, 0}, qlz[2] = {0, 0}, qhx[2] = {0, 0}, qhy[2] = {0, 0}, qhz[2] = {0, 0};
  uint32_t meta[2] = {0, 0}, imask = 0, off = 0;
  const uint32_t tb = tri_base[i];
  for (int sl = 0; sl < 8; ++sl) {
    const int k = by_slot[sl];
    if (k < 0) continue;
    const Kid& c = kids[k];
    const int w = sl >> 2, sh = 8 * (sl & 3);
    qlx[w] |= q_lo(lo.x, ex, c.lo.x) << sh;
    qly[w] |= q_lo(lo.y, ey, c.lo.y) << sh;
    qlz[w] |= q_lo(lo.z, ez, c.lo.z) << sh;
    qhx[w] |= q_hi(lo.x, ex, c.hi.x) << sh;
    qhy[w] |= q_hi(lo.y, ey, c.hi.y) << sh;
    qhz[w] |= q_hi(lo.z, ez, c.hi.z) << sh;
    if (!leaf_ref(c, as_leaf)) {
      imask |= 1u << sl;
      continue;
    }
    int pos, m;
    leaf_range(n2, c, cnt, first, &pos, &m);
    if (m < 1 || m > kBvh4MaxLeaf || off + (uint32_t)m > 32u || pos < 0 || pos + m > nt ||
        (long long)tb + off + m > nt) {
      atomicOr(err, kErrBadIndex);
      continue;
    }
    meta[w] |= (0x80u | ((uint32_t)(m - 1) << 5) | off) << sh;
    for (int t = 0; t < m; ++t)
      for (int q = 0; q < kTriF4; ++q)
        t8[(size_t)kTriF4 * (tb + off + t) + q] = tdfs[(size_t)kTriF4 * (pos + t) + q];
    off += (uint32_t)m;
  }
  const uint32_t eb = ((uint32_t)(ex & 0xff)) | ((uint32_t)(ey & 0xff) << 8) | ((uint32_t)(ez & 0xff) << 16) |
                      (imask << 24);
  uint4* o = n8 + (size_t)kNode8U4 * i;
  o[0] = make_uint4(__float_as_uint(lo.x), __float_as_uint(lo.y), __float_as_uint(lo.z), eb);
  o[1] = make_uint4(child_base[i], tb, meta[0], meta[1]);
  o[2] = make_uint4(qlx[0], qlx[1], qly[0], qly[1]);
  o[3] = make_uint4(qlz[0], qlz[1], qhx[0], qhx[1]);
  o[4] = make_uint4(qhy[0], qhy[1], qhz[0], qhz[1]);
}

unsigned blocks(long long n) { return (unsigned)((n + kB4Threads - 1) / kB4Threads); }

}  // namespace

size_t bvh4_scratch_bytes(int n_inner, int n_tris) { return b4_bytes(std::max(1, n_inner), std::max(1, n_tris)); }

namespace {

// The passes both collapses share: parents and reference counts, the tree
// check, the bottom-up SAH leaf decision and the depth-first positions.
// Returns 0, or -1 (*tree_ok = 0 for a malformed tree).
int prepare_tree(const float4* d_nodes2, int nn, int n_tris, const B4Scratch& b, int* tree_ok, int max_leaf,
                 cudaStream_t s) {
  cudaMemsetAsync(b.parent, 0xff, (size_t)nn * 4, s);
  cudaMemsetAsync(b.refs, 0, (size_t)nn * 4, s);
  cudaMemsetAsync(b.tri_refs, 0, (size_t)n_tris * 4, s);
  cudaMemsetAsync(b.counts, 0, 32, s);
  cudaMemsetAsync(b.err, 0, 4, s);
  cudaMemsetAsync(b.queue[0], 0, 4, s);  // level 1: the root
  parents_kernel<<<blocks(nn), kB4Threads, 0, s>>>(d_nodes2, nn, n_tris, b.parent, b.visit, b.is4, b.need, b.depth,
                                                    b.refs, b.tri_refs, b.err);
  verify_kernel<<<blocks(std::max(nn, n_tris)), kB4Threads, 0, s>>>(nn, n_tris, b.refs, b.tri_refs, b.err);
  uint32_t err = 0;
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  if (err != 0) {
    *tree_ok = 0;
    return -1;
  }
  *tree_ok = 1;
  bottom_up_kernel<<<blocks(nn), kB4Threads, 0, s>>>(d_nodes2, nn, b.parent, b.cnt, b.cost, b.as_leaf, b.dp_cost,
                                                      b.dp_split, b.visit, max_leaf, b.err);
  first_kernel<<<blocks(nn), kB4Threads, 0, s>>>(d_nodes2, nn, b.parent, b.cnt, b.first, b.counts + 4, b.err);
  return 0;
}

}  // namespace

int bvh4_plan(const float4* d_nodes2, int n_inner, int n_tris, void* scratch, Bvh4Plan* plan, cudaStream_t s,
              int max_leaf) {
  const int nn = n_inner;
  *plan = Bvh4Plan{};
  if (nn < 1 || n_tris < 2 || max_leaf < 1 || max_leaf > kBvh4MaxLeaf) return -1;
  B4Scratch b = b4_carve(scratch, nn, n_tris);
  if (prepare_tree(d_nodes2, nn, n_tris, b, &plan->tree_ok, max_leaf, s) != 0) return -1;
  uint32_t err = 0;
  int launches = 4;
  uint32_t n_in = 1;
  // one launch per 4-wide level; a tree has fewer levels than inner nodes
  for (int level = 0; n_in > 0; ++level) {
    if (level > nn) return -1;
    uint32_t* out_count = b.counts + ((level + 1) & 1);
    cudaMemsetAsync(out_count, 0, 4, s);
    mark_kernel<<<blocks(n_in), kB4Threads, 0, s>>>(d_nodes2, b.as_leaf, b.dp_cost, b.dp_split, b.queue[level & 1], n_in,
                                                    b.queue[(level + 1) & 1], out_count, b.is4, b.need, b.depth,
                                                    b.counts + 2);
    ++launches;
    if (cudaMemcpyAsync(&n_in, out_count, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -1;
  }
  launch_exclusive_scan(b.is4, b.slot, (size_t)nn, b.scan_tmp, s);
  launches += 3;
  uint32_t last[2] = {0, 0}, maxes[3] = {0, 0, 0};
  int root_cnt = 0;
  cudaMemcpyAsync(&last[0], b.slot + nn - 1, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&last[1], b.is4 + nn - 1, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(maxes, b.counts + 2, 12, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&root_cnt, b.cnt, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  if (err != 0 || root_cnt != n_tris) {
    plan->tree_ok = 0;
    return -1;
  }
  plan->depth2 = (int)maxes[2];
  plan->n_nodes4 = (int)(last[0] + last[1]);
  plan->stack_need = (int)maxes[0];
  plan->depth = (int)maxes[1];
  plan->launches = launches;
  return plan->n_nodes4;
}

int bvh4_emit(const float4* d_nodes2, const float4* d_tris2, int n_inner, int n_tris, void* scratch,
              float4* d_nodes4, float4* d_tris4, cudaStream_t s) {
  B4Scratch b = b4_carve(scratch, n_inner, n_tris);
  emit_kernel<<<blocks(n_inner), kB4Threads, 0, s>>>(d_nodes2, d_tris2, n_inner, n_tris, b.as_leaf, b.dp_cost,
                                                      b.dp_split, b.cnt, b.first, b.is4, b.slot, d_nodes4, d_tris4,
                                                      b.err);
  uint32_t err = 0;
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || err != 0) return -1;
  return 1;
}

// ---------------------------------------------------------------- 8-wide
namespace {

struct B8Extra {
  uint32_t* bfs;         // [nn] binary node of each 8-wide node (breadth-first order)
  uint32_t* child_base;  // [nn] first inner child of each 8-wide node
  uint32_t* tri_cnt;     // [nn] leaf triangles of each 8-wide node
  uint32_t* tri_base;    // [nn] their first position
  uint32_t* n_inner;     // [nn] per level: inner children of each node
  uint32_t* pos;         // [nn] per level: exclusive scan of n_inner
  uint32_t* q[2];        // [nn] level queues
  float4* tdfs;          // [nt * 3] triangles in depth-first order
};

size_t b8_extra_bytes(int nn, int nt) { return a256((size_t)nn * 4) * 8 + a256((size_t)nt * kTriF4 * 16); }

B8Extra b8_carve(void* scratch, int nn, int nt) {
  const size_t n = (size_t)nn;
  char* p = static_cast<char*>(scratch) + b4_bytes(nn, nt);
  B8Extra x;
  x.bfs = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.child_base = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.tri_cnt = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.tri_base = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.n_inner = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.pos = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.q[0] = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.q[1] = reinterpret_cast<uint32_t*>(p); p += a256(n * 4);
  x.tdfs = reinterpret_cast<float4*>(p);
  return x;
}

}  // namespace

size_t bvh8_scratch_bytes(int n_inner, int n_tris) {
  const int nn = std::max(1, n_inner), nt = std::max(1, n_tris);
  return b4_bytes(nn, nt) + b8_extra_bytes(nn, nt);
}

int bvh8_plan(const float4* d_nodes2, int n_inner, int n_tris, void* scratch, Bvh8Plan* plan, cudaStream_t s) {
  const int nn = n_inner;
  *plan = Bvh8Plan{};
  if (nn < 1 || n_tris < 2) return -1;
  B4Scratch b = b4_carve(scratch, nn, n_tris);
  B8Extra x = b8_carve(scratch, nn, n_tris);
  if (prepare_tree(d_nodes2, nn, n_tris, b, &plan->tree_ok, kBvh4MaxLeaf, s) != 0) return -1;
  int launches = 4;
  cudaMemsetAsync(x.q[0], 0, 4, s);  // level 0: the root
  uint32_t n_in = 1, base = 0;
  int depth = 0;
  // one level per round; node numbers are breadth first, so each node's
  // inner children are consecutive
  while (n_in > 0) {
    if (depth > nn) return -1;
    const uint32_t* q_in = x.q[depth & 1];
    count8_kernel<<<blocks(n_in), kB4Threads, 0, s>>>(d_nodes2, b.as_leaf, b.cnt, b.first, q_in, n_in, base, x.n_inner,
                                                      x.tri_cnt, b.err);
    launch_exclusive_scan(x.n_inner, x.pos, (size_t)n_in, b.scan_tmp, s);
    uint32_t last[2] = {0, 0};
    cudaMemcpyAsync(&last[0], x.n_inner + n_in - 1, 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&last[1], x.pos + n_in - 1, 4, cudaMemcpyDeviceToHost, s);
    place8_kernel<<<blocks(n_in), kB4Threads, 0, s>>>(d_nodes2, b.as_leaf, q_in, n_in, x.pos, base, base + n_in,
                                                      x.q[(depth + 1) & 1], x.bfs, x.child_base);
    launches += 5;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    base += n_in;
    n_in = last[0] + last[1];
    if ((size_t)base + n_in > (size_t)nn) return -1;
    ++depth;
  }
  launch_exclusive_scan(x.tri_cnt, x.tri_base, (size_t)base, b.scan_tmp, s);
  launches += 3;
  uint32_t tl[2] = {0, 0}, err = 0;
  cudaMemcpyAsync(&tl[0], x.tri_cnt + base - 1, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&tl[1], x.tri_base + base - 1, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  if (err != 0 || tl[0] + tl[1] != (uint32_t)n_tris) {
    plan->tree_ok = 0;
    return -1;
  }
  plan->n_nodes8 = (int)base;
  plan->depth = depth;
  plan->launches = launches;
  return plan->n_nodes8;
}

int bvh8_emit(const float4* d_nodes2, const float4* d_tris2, int n_inner, int n_tris, void* scratch, int n_nodes8,
              uint4* d_nodes8, float4* d_tris8, cudaStream_t s) {
  B4Scratch b = b4_carve(scratch, n_inner, n_tris);
  B8Extra x = b8_carve(scratch, n_inner, n_tris);
  relayout_kernel<<<blocks(n_inner), kB4Threads, 0, s>>>(d_nodes2, d_tris2, n_inner, n_tris, b.cnt, b.first, x.tdfs,
                                                          b.err);
  emit8_kernel<<<blocks(n_nodes8), kB4Threads, 0, s>>>(d_nodes2, (uint32_t)n_nodes8, b.as_leaf, b.cnt, b.first, x.bfs,
                                                        x.child_base, x.tri_base, x.tdfs, n_tris, d_nodes8, d_tris8,
                                                        b.err);
  uint32_t err = 0;
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || err != 0) return -1;
  return 1;
}

// ---------------------------------------------------------------- two-level
namespace {

// links of n 4-wide nodes: inner links += node_off, leaf ranges moved by
// tri_off (the nodes joined to a concatenation)
__global__ void link_offset_kernel(float4* __restrict__ n4, int n, int node_off, int tri_off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int4* l = reinterpret_cast<int4*>(n4 + (size_t)kNode4F4 * i + 6);
  int4 v = *l;
  int* c[4] = {&v.x, &v.y, &v.z, &v.w};
  for (int k = 0; k < 4; ++k) {
    if (*c[k] == kBvh4Empty) continue;
    if (*c[k] >= 0) *c[k] += node_off;
    else *c[k] = leaf_code(leaf_first(*c[k]) + tri_off, leaf_count(*c[k]));
  }
  *l = v;
}

// TLAS leaves (one record each) point at the instance itself
__global__ void tlas_leaf_kernel(float4* __restrict__ n4, int n, const float4* __restrict__ t4, int n_inst,
                                 uint32_t* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int4* l = reinterpret_cast<int4*>(n4 + (size_t)kNode4F4 * i + 6);
  int4 v = *l;
  int* c[4] = {&v.x, &v.y, &v.z, &v.w};
  for (int k = 0; k < 4; ++k) {
    if (*c[k] == kBvh4Empty || *c[k] >= 0) continue;
    if (leaf_count(*c[k]) != 1 || leaf_first(*c[k]) >= n_inst) {
      atomicOr(err, kErrBadIndex);
      continue;
    }
    const int inst = __float_as_int(t4[(size_t)kTriF4 * leaf_first(*c[k])].w);
    if (inst < 0 || inst >= n_inst) atomicOr(err, kErrBadIndex);
    *c[k] = leaf_code(inst, 1);
  }
  *l = v;
}

}  // namespace

void launch_link_offset(float4* nodes4, int n, int node_off, int tri_off, cudaStream_t s) {
  if (n > 0) link_offset_kernel<<<blocks(n), kB4Threads, 0, s>>>(nodes4, n, node_off, tri_off);
}

void launch_tlas_leaves(float4* nodes4, int n, const float4* tris4, int n_inst, uint32_t* err, cudaStream_t s) {
  if (n > 0) tlas_leaf_kernel<<<blocks(n), kB4Threads, 0, s>>>(nodes4, n, tris4, n_inst, err);
}

// ---------------------------------------------------------------- SAH cost
namespace {

// per 4-wide node: the surface areas of its inner children (each a node
// step) and of its leaves times their triangle counts (triangle tests)
__global__ void sah4_kernel(const float4* __restrict__ n4, int n, float* __restrict__ node_a,
                            float* __restrict__ tri_a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4* nb = n4 + (size_t)kNode4F4 * i;
  const float4 lx = nb[0], hx = nb[1], ly = nb[2], hy = nb[3], lz = nb[4], hz = nb[5];
  const int4 ch = *reinterpret_cast<const int4*>(nb + 6);
  const float lo[3][4] = {{lx.x, lx.y, lx.z, lx.w}, {ly.x, ly.y, ly.z, ly.w}, {lz.x, lz.y, lz.z, lz.w}};
  const float hi[3][4] = {{hx.x, hx.y, hx.z, hx.w}, {hy.x, hy.y, hy.z, hy.w}, {hz.x, hz.y, hz.z, hz.w}};
  const int c[4] = {ch.x, ch.y, ch.z, ch.w};
  float na = 0.0f, ta = 0.0f;
  for (int k = 0; k < 4; ++k) {
    if (c[k] == kBvh4Empty) continue;
    const float a = box_area(f3(lo[0][k], lo[1][k], lo[2][k]), f3(hi[0][k], hi[1][k], hi[2][k]));
    if (c[k] >= 0) na += a;
    else ta += a * (float)leaf_count(c[k]);
  }
  node_a[i] = na;
  tri_a[i] = ta;
}

}  // namespace

int bvh4_sah(const float4* d_nodes4, int n4, cudaStream_t s, double* node_term, double* tri_term) {
  *node_term = *tri_term = 0.0;
  if (n4 < 1) return -1;
  const int grid = (n4 + step_block_size() - 1) / step_block_size();  // launch_block_sums' partial sums
  float* fa = nullptr;
  double* da = nullptr;
  if (cudaMalloc(&fa, 8 * (size_t)n4) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (cudaMalloc(&da, 8 * (size_t)(2 * grid + 2)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fa);
    return -1;
  }
  sah4_kernel<<<blocks(n4), kB4Threads, 0, s>>>(d_nodes4, n4, fa, fa + n4);
  launch_block_sums(fa, (unsigned long long)n4, da, s);
  launch_sum_doubles(da, grid, da + 2 * grid, s);
  launch_block_sums(fa + n4, (unsigned long long)n4, da + grid, s);
  launch_sum_doubles(da + grid, grid, da + 2 * grid + 1, s);
  double sums[2] = {0.0, 0.0};
  float4 root[kNode4F4];
  cudaMemcpyAsync(sums, da + 2 * grid, 16, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(root, d_nodes4, sizeof(root), cudaMemcpyDeviceToHost, s);
  const bool ok = cudaStreamSynchronize(s) == cudaSuccess;
  cudaFree(fa);
  cudaFree(da);
  if (!ok) return -1;
  // the root box: the union of the root node's children
  const float* lo[3] = {&root[0].x, &root[2].x, &root[4].x};
  const float* hi[3] = {&root[1].x, &root[3].x, &root[5].x};
  const int* links = reinterpret_cast<const int*>(&root[6]);
  double bl[3] = {1e300, 1e300, 1e300}, bh[3] = {-1e300, -1e300, -1e300};
  for (int k = 0; k < 4; ++k) {
    if (links[k] == kBvh4Empty) continue;
    for (int a = 0; a < 3; ++a) {
      bl[a] = std::min(bl[a], (double)lo[a][k]);
      bh[a] = std::max(bh[a], (double)hi[a][k]);
    }
  }
  const double dx = bh[0] - bl[0], dy = bh[1] - bl[1], dz = bh[2] - bl[2];
  const double a0 = 2.0 * (dx * dy + dy * dz + dz * dx);
  if (!(a0 > 0.0)) return -1;
  *node_term = 1.0 + sums[0] / a0;
  *tri_term = sums[1] / a0;
  return 1;
}

}  // namespace dr
