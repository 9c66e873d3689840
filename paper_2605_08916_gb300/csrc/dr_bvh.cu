// BVH construction on the GPU (linear BVH: Morton codes of triangle
// centroids, radix sort, Karras 2012 "Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees" hierarchy emission, then a
// bottom-up box pass).  The paper uses the graphics API's hardware
// acceleration structure (Sec. 4.3); this replaces it for software traversal.
#include "dr_internal.h"

namespace dr {

namespace {

constexpr int kB = 256;

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

struct BvhScratch {
  uint2* keys0;     // (morton, tri)
  uint2* keys1;
  float* cbox;      // per block centroid bounds partials: 6 floats
  float* gbox;      // 6 floats: global centroid bounds
  int* parent;      // 2n - 1 (internal 0..n-2, leaves n-1..2n-2)
  int* child;       // 2 per internal node (encoded: >= 0 internal, leaf -> n - 1 + k)
  float* box;       // 6 floats per node (internal + leaf), [2n - 1][6]
  unsigned* flag;   // n - 1
  void* sort_scratch;
};

BvhScratch carve(void* p, int n) {
  BvhScratch s;
  char* c = static_cast<char*>(p);
  const size_t nn = (size_t)n;
  const int nblk = (n + kB - 1) / kB;
  s.keys0 = reinterpret_cast<uint2*>(c); c += a256(nn * 8);
  s.keys1 = reinterpret_cast<uint2*>(c); c += a256(nn * 8);
  s.cbox = reinterpret_cast<float*>(c); c += a256((size_t)nblk * 6 * 4);
  s.gbox = reinterpret_cast<float*>(c); c += a256(6 * 4);
  s.parent = reinterpret_cast<int*>(c); c += a256((2 * nn) * 4);
  s.child = reinterpret_cast<int*>(c); c += a256((2 * nn) * 4);
  s.box = reinterpret_cast<float*>(c); c += a256((2 * nn) * 6 * 4);
  s.flag = reinterpret_cast<unsigned*>(c); c += a256(nn * 4);
  s.sort_scratch = c;
  return s;
}

DR_D float3 vtx(const float* v, int i) { return f3(v[3 * i], v[3 * i + 1], v[3 * i + 2]); }

__global__ void centroid_bounds_kernel(const float* __restrict__ verts, const int* __restrict__ tris, int n,
                                       float* __restrict__ partial) {
  __shared__ float sh[6][kB];
  const int i = blockIdx.x * kB + threadIdx.x;
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  if (i < n) {
    const float3 c = (vtx(verts, tris[3 * i]) + vtx(verts, tris[3 * i + 1]) + vtx(verts, tris[3 * i + 2])) * (1.0f / 3.0f);
    lo[0] = hi[0] = c.x; lo[1] = hi[1] = c.y; lo[2] = hi[2] = c.z;
  }
  for (int a = 0; a < 3; ++a) { sh[a][threadIdx.x] = lo[a]; sh[3 + a][threadIdx.x] = hi[a]; }
  __syncthreads();
  for (int o = kB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int a = 0; a < 3; ++a) {
        sh[a][threadIdx.x] = fminf(sh[a][threadIdx.x], sh[a][threadIdx.x + o]);
        sh[3 + a][threadIdx.x] = fmaxf(sh[3 + a][threadIdx.x], sh[3 + a][threadIdx.x + o]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) partial[blockIdx.x * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// One block: the union of the nblk partial boxes (min / max are exact, so
// the order of the reduction does not matter).
__global__ void bounds_final_kernel(const float* __restrict__ partial, int nblk, float* __restrict__ out) {
  __shared__ float sh[6][kB];
  float v[6] = {3.4e38f, 3.4e38f, 3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int a = 0; a < 6; ++a) v[a] = a < 3 ? fminf(v[a], partial[b * 6 + a]) : fmaxf(v[a], partial[b * 6 + a]);
  for (int a = 0; a < 6; ++a) sh[a][threadIdx.x] = v[a];
  __syncthreads();
  for (int o = kB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int a = 0; a < 6; ++a)
        sh[a][threadIdx.x] = a < 3 ? fminf(sh[a][threadIdx.x], sh[a][threadIdx.x + o])
                                   : fmaxf(sh[a][threadIdx.x], sh[a][threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

DR_D uint32_t expand10(uint32_t v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void morton_kernel(const float* __restrict__ verts, const int* __restrict__ tris, int n,
                              const float* __restrict__ gbox, uint2* __restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float3 c = (vtx(verts, tris[3 * i]) + vtx(verts, tris[3 * i + 1]) + vtx(verts, tris[3 * i + 2])) * (1.0f / 3.0f);
  const float lo[3] = {gbox[0], gbox[1], gbox[2]}, hi[3] = {gbox[3], gbox[4], gbox[5]};
  const float cc[3] = {c.x, c.y, c.z};
  uint32_t q[3];
  for (int a = 0; a < 3; ++a) {
    const float ext = hi[a] - lo[a];
    float u = ext > 0.0f ? (cc[a] - lo[a]) / ext : 0.5f;
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    q[a] = (uint32_t)fminf(u * 1024.0f, 1023.0f);
  }
  keys[i] = make_uint2((expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]), (uint32_t)i);
}

// common-prefix length of sorted keys i, j (ties broken by index)
DR_D int delta(const uint2* __restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = k[i].x, b = k[j].x;
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void hierarchy_kernel(const uint2* __restrict__ k, int n, int* __restrict__ child, int* __restrict__ parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int dirn = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(k, n, i, i - dirn);
  int lmax = 2;
  while (delta(k, n, i, i + lmax * dirn) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(k, n, i, i + (l + t) * dirn) > dmin) l += t;
  const int j = i + l * dirn;
  const int dnode = delta(k, n, i, j);
  // binary search for the split; t halves (rounding up) until it reaches 1,
  // and a degenerate l = 0 exits after one pass
  int s = 0;
  int t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(k, n, i, i + (s + t) * dirn) > dnode) s += t;
  } while (t > 1);
  const int g = i + s * dirn + min(dirn, 0);
  const int lo = min(i, j), hi = max(i, j);
  const int left = lo == g ? (n - 1) + g : g;
  const int right = hi == g + 1 ? (n - 1) + g + 1 : g + 1;
  child[2 * i] = left;
  child[2 * i + 1] = right;
  parent[left] = i;
  parent[right] = i;
}

__global__ void leaf_boxes_kernel(const float* __restrict__ verts, const int* __restrict__ tris,
                                  const uint2* __restrict__ k, int n, float* __restrict__ box,
                                  float4* __restrict__ tri_out, unsigned* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) flag[i] = 0u;
  if (i >= n) return;
  const int t = (int)k[i].y;
  const float3 v0 = vtx(verts, tris[3 * t]), v1 = vtx(verts, tris[3 * t + 1]), v2 = vtx(verts, tris[3 * t + 2]);
  float* b = box + (size_t)(n - 1 + i) * 6;
  b[0] = fminf(v0.x, fminf(v1.x, v2.x)); b[1] = fminf(v0.y, fminf(v1.y, v2.y)); b[2] = fminf(v0.z, fminf(v1.z, v2.z));
  b[3] = fmaxf(v0.x, fmaxf(v1.x, v2.x)); b[4] = fmaxf(v0.y, fmaxf(v1.y, v2.y)); b[5] = fmaxf(v0.z, fmaxf(v1.z, v2.z));
  const float3 e1 = v1 - v0, e2 = v2 - v0;
  tri_out[3 * i + 0] = make_float4(v0.x, v0.y, v0.z, __int_as_float(t));
  tri_out[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, 0.0f);
  tri_out[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, 0.0f);
}

// Bottom-up boxes: the second child to arrive at a node computes its box.
__global__ void internal_boxes_kernel(int n, const int* __restrict__ child, const int* __restrict__ parent,
                                      float* box, unsigned* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int node = n - 1 + i;
  // a leaf is at most n - 1 levels deep; the cap only guards a corrupt tree
  for (int guard = 0; node != 0 && guard < n; ++guard) {
    const int p = parent[node];
    if (p < 0 || p >= n - 1) return;
    __threadfence();
    if (atomicAdd(&flag[p], 1u) == 0u) return;
    __threadfence();
    const int a = child[2 * p], b = child[2 * p + 1];
    volatile float* ba = box + (size_t)a * 6;
    volatile float* bb = box + (size_t)b * 6;
    float* bp = box + (size_t)p * 6;
    for (int q = 0; q < 3; ++q) {
      bp[q] = fminf(ba[q], bb[q]);
      bp[3 + q] = fmaxf(ba[3 + q], bb[3 + q]);
    }
    node = p;
  }
}

__global__ void emit_nodes_kernel(int n, const int* __restrict__ child, const float* __restrict__ box,
                                  float4* __restrict__ nodes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int a = child[2 * i], b = child[2 * i + 1];
  const float* ba = box + (size_t)a * 6;
  const float* bb = box + (size_t)b * 6;
  const int ca = a >= n - 1 ? leaf_code(a - (n - 1), 1) : a;
  const int cb = b >= n - 1 ? leaf_code(b - (n - 1), 1) : b;
  nodes[4 * i + 0] = make_float4(ba[0], ba[1], ba[2], ba[3]);
  nodes[4 * i + 1] = make_float4(ba[4], ba[5], bb[0], bb[1]);
  nodes[4 * i + 2] = make_float4(bb[2], bb[3], bb[4], bb[5]);
  nodes[4 * i + 3] = make_float4(__int_as_float(ca), __int_as_float(cb), 0.0f, 0.0f);
}

// single triangle: root with one leaf child and one empty box
__global__ void single_root_kernel(const float* __restrict__ verts, const int* __restrict__ tris,
                                   float4* __restrict__ nodes, float4* __restrict__ tri_out) {
  const float3 v0 = vtx(verts, tris[0]), v1 = vtx(verts, tris[1]), v2 = vtx(verts, tris[2]);
  const float3 lo = f3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
  const float3 hi = f3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
  const float inf = __int_as_float(0x7f800000);
  nodes[0] = make_float4(lo.x, lo.y, lo.z, hi.x);
  nodes[1] = make_float4(hi.y, hi.z, inf, inf);
  nodes[2] = make_float4(inf, -inf, -inf, -inf);
  nodes[3] = make_float4(__int_as_float(leaf_code(0, 1)), __int_as_float(leaf_code(0, 1)), 0.0f, 0.0f);
  const float3 e1 = v1 - v0, e2 = v2 - v0;
  tri_out[0] = make_float4(v0.x, v0.y, v0.z, __int_as_float(0));
  tri_out[1] = make_float4(e1.x, e1.y, e1.z, 0.0f);
  tri_out[2] = make_float4(e2.x, e2.y, e2.z, 0.0f);
}

// Surface record of each triangle; flag bit 0 of s2.w = shading normals
// (all three vertex normals non-zero).
__global__ void surface_kernel(const float* __restrict__ verts, const int* __restrict__ tris,
                               const int* __restrict__ tri_mat, const float* __restrict__ sel,
                               const float* __restrict__ vn, int n, float4* __restrict__ surf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float3 v0 = vtx(verts, tris[3 * i]), v1 = vtx(verts, tris[3 * i + 1]), v2 = vtx(verts, tris[3 * i + 2]);
  const float3 e1 = v1 - v0, e2 = v2 - v0;
  const float3 N = cross(e1, e2);
  const float nn = dot(N, N);
  const float3 ng = N * rsqrtf(nn);
  const float3 au = cross(e2, N) * (1.0f / nn);
  const float3 av = cross(N, e1) * (1.0f / nn);
  surf[5 * i + 0] = make_float4(v0.x, v0.y, v0.z, __int_as_float(tri_mat[i]));
  surf[5 * i + 1] = make_float4(N.x, N.y, N.z, 0.5f * sqrtf(nn));
  int flags = 0;
  if (vn) {
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
      const int v = tris[3 * i + k];
      ok = ok && (vn[3 * v] != 0.0f || vn[3 * v + 1] != 0.0f || vn[3 * v + 2] != 0.0f);
    }
    flags |= ok ? 1 : 0;
  }
  surf[5 * i + 2] = make_float4(ng.x, ng.y, ng.z, __int_as_float(flags));
  surf[5 * i + 3] = make_float4(au.x, au.y, au.z, sel ? sel[i] : 0.0f);
  surf[5 * i + 4] = make_float4(av.x, av.y, av.z, 0.0f);
}

__global__ void gather_normals_kernel(const float* __restrict__ vn, const int* __restrict__ tris, int n,
                                      float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 3; ++k) {
    const int v = tris[3 * i + k];
    out[9 * i + 3 * k + 0] = vn[3 * v + 0];
    out[9 * i + 3 * k + 1] = vn[3 * v + 1];
    out[9 * i + 3 * k + 2] = vn[3 * v + 2];
  }
}

// ---------------------------------------------------------------- PLOC
// Parallel locally-ordered clustering (Meister and Bittner 2018): clusters
// kept in Morton order; each finds the neighbour within +-r whose merged box
// has the smallest surface area; mutual nearest neighbours merge; the
// cluster list is compacted; repeat until one cluster remains.  Inner nodes
// are numbered from the top (the last merge is node 0, the root), so the
// hierarchy has the same layout as the linear build.

DR_D float box_area(const float* a, const float* b) {
  const float dx = fmaxf(a[3], b[3]) - fminf(a[0], b[0]);
  const float dy = fmaxf(a[4], b[4]) - fminf(a[1], b[1]);
  const float dz = fmaxf(a[5], b[5]) - fminf(a[2], b[2]);
  return dx * dy + dy * dz + dz * dx;
}

__global__ void ploc_init_kernel(int n, const float* __restrict__ box, int* __restrict__ cl_node,
                                 float* __restrict__ cl_box, int* __restrict__ height) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cl_node[i] = n - 1 + i;
  height[n - 1 + i] = 1;
  for (int q = 0; q < 6; ++q) cl_box[6 * i + q] = box[(size_t)(n - 1 + i) * 6 + q];
}

// The clustering loop keeps its state on the device, so that the host
// enqueues several passes between synchronisations:
//   st[0] = m, clusters left; st[1] = inner nodes created so far;
//   st[2] = merges of the current pass; st[3] = height of the tallest
//   subtree built so far (a leaf: 1).
// Grids are sized by the host's upper bound m_ub >= m; a pass that finds
// m = 1 copies the single cluster and changes nothing.
constexpr int kPlocM = 0, kPlocCreated = 1, kPlocMerges = 2, kPlocMaxH = 3, kPlocState = 4;

__global__ void ploc_nn_kernel(const int* __restrict__ st, int r, const float* __restrict__ cl_box,
                               int* __restrict__ nn) {
  const int m = st[kPlocM];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  float bi[6];
  for (int q = 0; q < 6; ++q) bi[q] = cl_box[6 * i + q];
  float best = __int_as_float(0x7f800000);
  int bj = i == 0 ? 1 : i - 1;
  const int lo = max(0, i - r), hi = min(m - 1, i + r);
  for (int j = lo; j <= hi; ++j) {
    if (j == i) continue;
    float bb[6];
    for (int q = 0; q < 6; ++q) bb[q] = cl_box[6 * j + q];
    const float a = box_area(bi, bb);
    if (a < best) {  // first minimum wins: ties go to the smaller index
      best = a;
      bj = j;
    }
  }
  nn[i] = bj;
}

// flag[i] = 1 for the left cluster of each mutual nearest-neighbour pair;
// zero from m up to m_ub, so that a scan over m_ub entries counts the pass
__global__ void ploc_flag_kernel(const int* __restrict__ st, int m_ub, const int* __restrict__ nn,
                                 uint32_t* __restrict__ flag) {
  const int m = st[kPlocM];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m_ub) return;
  if (i >= m) {
    flag[i] = 0u;
    return;
  }
  const int j = nn[i];
  flag[i] = (j >= 0 && j < m && nn[j] == i && i < j) ? 1u : 0u;
}

// The pass's merge count (scan of the flags); when no mutual pair exists
// (degenerate ties) clusters 0 and 1 merge instead.  All flags are zero
// then, so the scan is zero everywhere, which is what the merge of cluster
// 0 needs.
__global__ void ploc_count_kernel(int* __restrict__ st, int* __restrict__ nn, uint32_t* __restrict__ flag,
                                  const uint32_t* __restrict__ pos) {
  const int m = st[kPlocM];
  if (m <= 1) {
    st[kPlocMerges] = 0;
    return;
  }
  int merges = (int)(pos[m - 1] + flag[m - 1]);
  if (merges == 0) {
    nn[0] = 1;
    nn[1] = 0;
    flag[0] = 1u;
    flag[1] = 0u;
    merges = 1;
  }
  st[kPlocMerges] = merges;
}

// Merges the flagged pairs: the k-th merge (k = exclusive scan of the flags)
// creates inner node (n - 2 - created) - k.  Writes the surviving cluster
// list's keep flags (1 = keep) into keep, zero from m up to m_ub.
__global__ void ploc_merge_kernel(int* __restrict__ st, int n, int m_ub, const int* __restrict__ nn,
                                  const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                  int* __restrict__ cl_node, float* __restrict__ cl_box, int* __restrict__ child,
                                  float* __restrict__ box, uint32_t* __restrict__ keep, int* __restrict__ height) {
  const int m = st[kPlocM];
  const int base = (n - 2) - st[kPlocCreated];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m_ub) return;
  if (i >= m) {
    keep[i] = 0u;
    return;
  }
  const int j = nn[i];
  const bool merging_left = flag[i] != 0u;
  const bool merged_away = j >= 0 && j < m && flag[j] != 0u && nn[j] == i;  // i is the right partner of j
  keep[i] = merged_away ? 0u : 1u;
  if (!merging_left) return;
  const int idx = base - (int)pos[i];
  const int a = cl_node[i], b = cl_node[j];
  child[2 * idx] = a;
  child[2 * idx + 1] = b;
  const int h = max(height[a], height[b]) + 1;
  height[idx] = h;
  atomicMax(&st[kPlocMaxH], h);
  float u[6];
  for (int q = 0; q < 3; ++q) {
    u[q] = fminf(cl_box[6 * i + q], cl_box[6 * j + q]);
    u[3 + q] = fmaxf(cl_box[6 * i + 3 + q], cl_box[6 * j + 3 + q]);
  }
  for (int q = 0; q < 6; ++q) {
    box[(size_t)idx * 6 + q] = u[q];
    cl_box[6 * i + q] = u[q];
  }
  cl_node[i] = idx;
}

__global__ void ploc_compact_kernel(const int* __restrict__ st, const uint32_t* __restrict__ keep,
                                    const uint32_t* __restrict__ pos, const int* __restrict__ cl_node,
                                    const float* __restrict__ cl_box, int* __restrict__ out_node,
                                    float* __restrict__ out_box) {
  const int m = st[kPlocM];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || !keep[i]) return;
  const int o = (int)pos[i];
  out_node[o] = cl_node[i];
  for (int q = 0; q < 6; ++q) out_box[6 * o + q] = cl_box[6 * i + q];
}

// end of a pass: m -= merges, created += merges
__global__ void ploc_advance_kernel(int* __restrict__ st) {
  st[kPlocCreated] += st[kPlocMerges];
  st[kPlocM] -= st[kPlocMerges];
}

__global__ void ploc_state_init_kernel(int* __restrict__ st, int n) {
  st[kPlocM] = n;
  st[kPlocCreated] = 0;
  st[kPlocMerges] = 0;
  st[kPlocMaxH] = 1;
}

}  // namespace

size_t ploc_scratch_bytes(int nt) {
  const size_t n = (size_t)(nt < 2 ? 2 : nt);
  return a256(n * 4) * 2 + a256(n * 24) * 2 + a256(n * 4) * 4 + a256(kPlocState * 4) + a256(2 * n * 4) +
         scan_scratch_bytes(n) + 256;
}

int build_ploc(const float* d_verts, const int* d_tris, int n, float4* d_nodes, float4* d_tris_out, void* scratch,
               void* ploc_scratch, int radius, int max_height, cudaStream_t st) {
  if (n <= 1) return build_lbvh(d_verts, d_tris, n, d_nodes, d_tris_out, scratch, st);
  BvhScratch s = carve(scratch, n);
  const int nblk = (n + kB - 1) / kB;
  centroid_bounds_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, n, s.cbox);
  bounds_final_kernel<<<1, kB, 0, st>>>(s.cbox, nblk, s.gbox);
  morton_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, n, s.gbox, s.keys0);
  uint2* sorted = sort_pairs(s.keys0, s.keys1, (size_t)n, 32, s.sort_scratch, st);
  leaf_boxes_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, sorted, n, s.box, d_tris_out, s.flag);
  // carve the clustering buffers
  char* p = static_cast<char*>(ploc_scratch);
  const size_t nn_ = (size_t)n;
  int* node_a = reinterpret_cast<int*>(p); p += a256(nn_ * 4);
  int* node_b = reinterpret_cast<int*>(p); p += a256(nn_ * 4);
  float* box_a = reinterpret_cast<float*>(p); p += a256(nn_ * 24);
  float* box_b = reinterpret_cast<float*>(p); p += a256(nn_ * 24);
  int* nn = reinterpret_cast<int*>(p); p += a256(nn_ * 4);
  uint32_t* flag = reinterpret_cast<uint32_t*>(p); p += a256(nn_ * 4);
  uint32_t* pos = reinterpret_cast<uint32_t*>(p); p += a256(nn_ * 4);
  uint32_t* keep = reinterpret_cast<uint32_t*>(p); p += a256(nn_ * 4);
  int* state = reinterpret_cast<int*>(p); p += a256(kPlocState * 4);
  int* height = reinterpret_cast<int*>(p); p += a256(2 * nn_ * 4);  // per node id (inner, then leaves)
  void* scan_tmp = p;
  ploc_init_kernel<<<nblk, kB, 0, st>>>(n, s.box, node_a, box_a, height);
  ploc_state_init_kernel<<<1, 1, 0, st>>>(state, n);
  // every pass merges at least one pair, so at most n - 1 passes; the host
  // reads the cluster count back once per kPassesPerSync passes
  constexpr int kPassesPerSync = 6;
  int m_ub = n, passes = 0;
  int host[kPlocState] = {n, 0, 0, 0};
  while (host[kPlocM] > 1 && passes < n) {
    for (int q = 0; q < kPassesPerSync && passes < n; ++q, ++passes) {
      const int mb = (m_ub + kB - 1) / kB;
      ploc_nn_kernel<<<mb, kB, 0, st>>>(state, radius, box_a, nn);
      ploc_flag_kernel<<<mb, kB, 0, st>>>(state, m_ub, nn, flag);
      launch_exclusive_scan(flag, pos, (size_t)m_ub, scan_tmp, st);
      ploc_count_kernel<<<1, 1, 0, st>>>(state, nn, flag, pos);
      ploc_merge_kernel<<<mb, kB, 0, st>>>(state, n, m_ub, nn, flag, pos, node_a, box_a, s.child, s.box, keep,
                                           height);
      launch_exclusive_scan(keep, pos, (size_t)m_ub, scan_tmp, st);
      ploc_compact_kernel<<<mb, kB, 0, st>>>(state, keep, pos, node_a, box_a, node_b, box_b);
      ploc_advance_kernel<<<1, 1, 0, st>>>(state);
      std::swap(node_a, node_b);
      std::swap(box_a, box_b);
    }
    if (cudaMemcpyAsync(host, state, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    m_ub = std::max(host[kPlocM], 1);
  }
  if (host[kPlocM] != 1 || host[kPlocCreated] != n - 1) return -1;
  // exact ties among many boxes (coincident triangles, say) make every
  // cluster's nearest neighbour the same one, so that a pass merges a single
  // pair and the tree degenerates into a chain: too tall for the traversal
  // stack, the linear BVH (which orders equal Morton codes by index) is
  // built instead
  if (max_height > 0 && host[kPlocMaxH] > max_height)
    return build_lbvh(d_verts, d_tris, n, d_nodes, d_tris_out, scratch, st);
  emit_nodes_kernel<<<nblk, kB, 0, st>>>(n, s.child, s.box, d_nodes);
  return n - 1;
}

size_t bvh_scratch_bytes(int nt) {
  const size_t n = (size_t)(nt < 2 ? 2 : nt);
  const int nblk = (int)((n + kB - 1) / kB);
  return a256(n * 8) * 2 + a256((size_t)nblk * 24) + a256(24) + a256(2 * n * 4) * 2 + a256(2 * n * 24) +
         a256(n * 4) + sort_scratch_bytes(n);
}

int build_lbvh(const float* d_verts, const int* d_tris, int n, float4* d_nodes, float4* d_tris_out, void* scratch,
               cudaStream_t st) {
  if (n <= 0) return 0;
  if (n == 1) {
    single_root_kernel<<<1, 1, 0, st>>>(d_verts, d_tris, d_nodes, d_tris_out);
    return 1;
  }
  BvhScratch s = carve(scratch, n);
  const int nblk = (n + kB - 1) / kB;
  centroid_bounds_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, n, s.cbox);
  bounds_final_kernel<<<1, kB, 0, st>>>(s.cbox, nblk, s.gbox);
  morton_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, n, s.gbox, s.keys0);
  uint2* sorted = sort_pairs(s.keys0, s.keys1, (size_t)n, 32, s.sort_scratch, st);
  hierarchy_kernel<<<nblk, kB, 0, st>>>(sorted, n, s.child, s.parent);
  leaf_boxes_kernel<<<nblk, kB, 0, st>>>(d_verts, d_tris, sorted, n, s.box, d_tris_out, s.flag);
  internal_boxes_kernel<<<nblk, kB, 0, st>>>(n, s.child, s.parent, s.box, s.flag);
  emit_nodes_kernel<<<nblk, kB, 0, st>>>(n, s.child, s.box, d_nodes);
  return n - 1;
}

void launch_surface_records(const float* d_verts, const int* d_tris, const int* d_tri_mat, const float* d_sel,
                            const float* d_vnormals, int nt, float4* d_surf, cudaStream_t s) {
  if (nt <= 0) return;
  surface_kernel<<<(nt + kB - 1) / kB, kB, 0, s>>>(d_verts, d_tris, d_tri_mat, d_sel, d_vnormals, nt, d_surf);
}

void launch_gather_normals(const float* d_vnormals, const int* d_tris, int nt, float* d_tri_normals, cudaStream_t s) {
  if (nt <= 0) return;
  gather_normals_kernel<<<(nt + kB - 1) / kB, kB, 0, s>>>(d_vnormals, d_tris, nt, d_tri_normals);
}

}  // namespace dr
