// Collapse of the binary BVH into a 4-wide BVH, on the device, at scene
// upload.
//
// Leaves: a binary subtree of at most kBvh4MaxLeaf triangles becomes one
// leaf when the surface-area heuristic rates a leaf no more expensive than
// the subtree (unit cost per node visit and per triangle test, weighted by
// area relative to the parent).  Inner nodes: starting from a binary node's
// two children, the inner child of largest surface area is replaced by its
// own two children until there are four children or only leaves are left.
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
#include <algorithm>

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
  void* scan_tmp;
};

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

size_t b4_bytes(int nn, int nt) {
  const size_t n = (size_t)nn;
  return a256(n * 4) * 12 + a256((size_t)nt * 4) + a256(n) + a256(32) + a256(4) + a256(scan_scratch_bytes(n));
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

// settles node n (its inner children are settled): count, SAH cost, leaf
// decision
DR_D void settle(const float4* __restrict__ n2, int n, int* cnt, float* cost, uint8_t* as_leaf) {
  const Kid k0 = kid_of(n2, n, 0), k1 = kid_of(n2, n, 1);
  const float an = fmaxf(box_area(f3(fminf(k0.lo.x, k1.lo.x), fminf(k0.lo.y, k1.lo.y), fminf(k0.lo.z, k1.lo.z)),
                                  f3(fmaxf(k0.hi.x, k1.hi.x), fmaxf(k0.hi.y, k1.hi.y), fmaxf(k0.hi.z, k1.hi.z))),
                         1e-30f);
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
  const bool leaf = total <= kBvh4MaxLeaf && (float)total <= c_inner;
  cnt[n] = total;
  cost[n] = leaf ? (float)total : c_inner;
  as_leaf[n] = leaf ? 1 : 0;
}

// Each node with leaf links starts a walk towards the root; a node is
// settled by the walk that brings its second finished child, the first
// arrival ends its walk there.
__global__ void bottom_up_kernel(const float4* __restrict__ n2, int nn, const int* parent, int* cnt, float* cost,
                                 uint8_t* as_leaf, uint32_t* visit, uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const float4 d = n2[4 * n + 3];
  const uint32_t leaves = (__float_as_int(d.x) < 0 ? 1u : 0u) + (__float_as_int(d.y) < 0 ? 1u : 0u);
  if (leaves == 0) return;
  if (atomicAdd(&visit[n], leaves) + leaves < 2) return;
  __threadfence();
  int cur = n;
  for (int guard = 0; guard <= nn; ++guard) {
    settle(n2, cur, cnt, cost, as_leaf);
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

// greedy widening of binary node n to up to four children
DR_D int expand(const float4* __restrict__ n2, int n, const uint8_t* as_leaf, Kid kids[4]) {
  kids[0] = kid_of(n2, n, 0);
  kids[1] = kid_of(n2, n, 1);
  int nk = 2;
  while (nk < 4) {
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

__global__ void mark_kernel(const float4* __restrict__ n2, const uint8_t* as_leaf, const uint32_t* q_in, uint32_t n_in,
                            uint32_t* q_out, uint32_t* n_out, uint32_t* is4, int* need, int* depth, uint32_t* maxes) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_in) return;
  const int n = (int)q_in[t];
  Kid kids[4];
  const int nk = expand(n2, n, as_leaf, kids);
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

__global__ void emit_kernel(const float4* __restrict__ n2, const float4* __restrict__ t2, int nn, int nt,
                            const uint8_t* as_leaf, const int* cnt, const int* first, const uint32_t* is4,
                            const uint32_t* slot, float4* __restrict__ n4, float4* __restrict__ t4, uint32_t* err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const float4 dn = n2[4 * n + 3];
  // triangles of this node's binary leaf links, to their depth-first place
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
  if (!is4[n]) return;
  Kid kids[4];
  const int nk = expand(n2, n, as_leaf, kids);
  float lo[3][4] = {}, hi[3][4] = {};  // empty slots stay zero; the traversal skips them by their link
  int links[4] = {kBvh4Empty, kBvh4Empty, kBvh4Empty, kBvh4Empty};
  for (int k = 0; k < nk; ++k) {
    const Kid& c = kids[k];
    lo[0][k] = c.lo.x; lo[1][k] = c.lo.y; lo[2][k] = c.lo.z;
    hi[0][k] = c.hi.x; hi[1][k] = c.hi.y; hi[2][k] = c.hi.z;
    if (!leaf_ref(c, as_leaf)) {
      links[k] = (int)slot[c.code];
    } else if (c.code >= 0) {
      links[k] = leaf_code(first[c.code], cnt[c.code]);
    } else {
      const float4 d = n2[4 * c.parent + 3];
      const int pos = first[c.parent] + (c.side == 1 ? count_of(__float_as_int(d.x), cnt) : 0);
      links[k] = leaf_code(pos, leaf_count(c.code));
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

unsigned blocks(long long n) { return (unsigned)((n + kB4Threads - 1) / kB4Threads); }

}  // namespace

size_t bvh4_scratch_bytes(int n_inner, int n_tris) { return b4_bytes(std::max(1, n_inner), std::max(1, n_tris)); }

int bvh4_plan(const float4* d_nodes2, int n_inner, int n_tris, void* scratch, Bvh4Plan* plan, cudaStream_t s) {
  const int nn = n_inner;
  *plan = Bvh4Plan{};
  if (nn < 1 || n_tris < 2) return -1;
  B4Scratch b = b4_carve(scratch, nn, n_tris);
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
    plan->tree_ok = 0;
    return -1;
  }
  plan->tree_ok = 1;
  bottom_up_kernel<<<blocks(nn), kB4Threads, 0, s>>>(d_nodes2, nn, b.parent, b.cnt, b.cost, b.as_leaf, b.visit,
                                                      b.err);
  first_kernel<<<blocks(nn), kB4Threads, 0, s>>>(d_nodes2, nn, b.parent, b.cnt, b.first, b.counts + 4, b.err);
  int launches = 4;
  uint32_t n_in = 1;
  // one launch per 4-wide level; a tree has fewer levels than inner nodes
  for (int level = 0; n_in > 0; ++level) {
    if (level > nn) return -1;
    uint32_t* out_count = b.counts + ((level + 1) & 1);
    cudaMemsetAsync(out_count, 0, 4, s);
    mark_kernel<<<blocks(n_in), kB4Threads, 0, s>>>(d_nodes2, b.as_leaf, b.queue[level & 1], n_in,
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
  emit_kernel<<<blocks(n_inner), kB4Threads, 0, s>>>(d_nodes2, d_tris2, n_inner, n_tris, b.as_leaf, b.cnt, b.first,
                                                      b.is4, b.slot, d_nodes4, d_tris4, b.err);
  uint32_t err = 0;
  cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || err != 0) return -1;
  return 1;
}

}  // namespace dr
