// Internal launchers shared by the translation units of libdiffrestore.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dr_common.cuh"

namespace dr {

// Sets the thread-local message returned by dr_last_error().
void set_error_message(const char* msg);

// ---------------------------------------------------------------- sorting
// Stable LSD radix sort (8-bit digits) of 16-B splat records by pixel, or of
// 8-B (key, value) pairs by key.  `bits` = number of significant key bits.
// Scratch from sort_scratch_bytes(); no allocation inside.
size_t sort_scratch_bytes(size_t n);
// Sorts in[0..n) into out (in is used as the ping-pong buffer and is
// clobbered).  Returns a pointer to whichever buffer holds the result.
SplatRec* sort_splat_records(SplatRec* in, SplatRec* out, size_t n, int bits, void* scratch, cudaStream_t s);
// Device-wide exclusive scan of uint32 (out may alias in only if n <= one chunk).
size_t scan_scratch_bytes(size_t n);
void launch_exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, void* scratch, cudaStream_t s);
uint2* sort_pairs(uint2* in, uint2* out, size_t n, int bits, void* scratch, cudaStream_t s);

// accum[pix * 3 + c] += sum of the sorted records' values (FP64, in sorted
// order), one writer per pixel.  Records with pix >= n_pix are skipped and
// flagged in *err.
void launch_segment_reduce(const SplatRec* sorted, size_t n, double* accum, uint32_t n_pix, uint32_t* err,
                           cudaStream_t s);
// out[i] = k0 / tourCount * accum[i] (0 when tourCount == 0).
void launch_resolve(const double* accum, size_t n, const unsigned long long* tour_count, double k0, float* out,
                    cudaStream_t s);
// Resolve with the tour count given by value (replicas' merged counts).
void launch_resolve_count(const double* accum, size_t n, unsigned long long tour_count, double k0, float* out,
                          cudaStream_t s);

// ---------------------------------------------------------------- BVH
struct BvhBuildOut {
  int n_nodes;
};
// Builds the LBVH for nt triangles (verts [nv*3], tris [nt*3] on device)
// into nodes (4 float4 per node, nt - 1 nodes, at least 1) and leaf-ordered
// triangle records (3 float4 per triangle).  scratch: bvh_scratch_bytes(nt).
size_t bvh_scratch_bytes(int nt);
int build_lbvh(const float* d_verts, const int* d_tris, int nt, float4* d_nodes, float4* d_tris_out, void* scratch,
               cudaStream_t s);
// Same output layout, clustered by PLOC with search radius `radius`
// (second scratch of ploc_scratch_bytes(nt)).  Synchronises once per six
// clustering passes.  When the clustered tree is taller than max_height
// (root = 1; 0: no limit), which exact ties among many boxes can cause, the
// linear BVH is built into the same outputs instead.  Returns the node
// count, or -1 on failure.
size_t ploc_scratch_bytes(int nt);
int build_ploc(const float* d_verts, const int* d_tris, int nt, float4* d_nodes, float4* d_tris_out, void* scratch,
               void* ploc_scratch, int radius, int max_height, cudaStream_t s);
// Per-triangle surface records (5 float4) from the device arrays; sel is
// the light-selection probability per triangle (device, may be null).
void launch_surface_records(const float* d_verts, const int* d_tris, const int* d_tri_mat, const float* d_sel,
                            const float* d_vnormals, int nt, float4* d_surf, cudaStream_t s);
void launch_gather_normals(const float* d_vnormals, const int* d_tris, int nt, float* d_tri_normals,
                           cudaStream_t s);
// Device-side collapse of the binary BVH (4 float4 per node, n_inner nodes;
// triangles 3 float4 each) into the 4-wide layout, triangles re-laid in
// depth-first order.  bvh4_plan runs every pass but the output (one
// synchronisation per 4-wide level) and returns the 4-wide node count, or -1
// (bad tree, fewer than 2 triangles, CUDA error); bvh4_emit then writes
// nodes4 [count * 7] and tris4 [n_tris * 3] (returns 1, or -1).  Both use
// the same scratch of bvh4_scratch_bytes(n_inner).
struct Bvh4Plan {
  int n_nodes4, depth, stack_need, launches;
  int tree_ok;  // 1: every inner node but the root and every triangle referenced exactly once
  int depth2;   // height of the binary tree (root = 1)
};
size_t bvh4_scratch_bytes(int n_inner, int n_tris);
int bvh4_plan(const float4* d_nodes2, int n_inner, int n_tris, void* scratch, Bvh4Plan* plan, cudaStream_t s,
              int max_leaf = kBvh4MaxLeaf);
int bvh4_emit(const float4* d_nodes2, const float4* d_tris2, int n_inner, int n_tris, void* scratch,
              float4* d_nodes4, float4* d_tris4, cudaStream_t s);
// The same collapse to the 8-wide compressed layout (kNode8U4): nodes in
// breadth-first order (one synchronisation per level), each node's leaf
// triangles consecutive.  bvh8_plan returns the node count (or -1);
// bvh8_emit writes nodes8 [count * 5 uint4] and tris8 [n_tris * 3].
struct Bvh8Plan {
  int n_nodes8, depth, launches;
  int tree_ok;
};
size_t bvh8_scratch_bytes(int n_inner, int n_tris);
int bvh8_plan(const float4* d_nodes2, int n_inner, int n_tris, void* scratch, Bvh8Plan* plan, cudaStream_t s);
int bvh8_emit(const float4* d_nodes2, const float4* d_tris2, int n_inner, int n_tris, void* scratch, int n_nodes8,
              uint4* d_nodes8, float4* d_tris8, cudaStream_t s);
// Two-level BVH assembly: shift the links of n 4-wide nodes by node_off /
// tri_off (BLAS concatenation), and turn TLAS leaves (one record each) into
// instance indices read from the records' ids.
void launch_link_offset(float4* nodes4, int n, int node_off, int tri_off, cudaStream_t s);
// Surface-area-heuristic cost of a 4-wide BVH for a ray that hits the root
// box (a box is entered with probability area / root area): expected node
// steps (*node_term, the root's included) and triangle tests (*tri_term).
// Returns 1, or -1.  Synchronises.
int bvh4_sah(const float4* d_nodes4, int n4, cudaStream_t s, double* node_term, double* tri_term);
void launch_tlas_leaves(float4* nodes4, int n, const float4* tris4, int n_inst, uint32_t* err, cudaStream_t s);

// ---------------------------------------------------------------- chains
enum Drift { kDriftNone = 0, kDriftFD = 1, kDriftAdjoint = 2, kDriftMala = 3 };

// What a replayed CUDA graph reads from device memory instead of its
// captured launch arguments, so that one graph serves every step, seed,
// frame and k0: the step index (advanced on the device after each step),
// the Philox key and frame, and the killing-rate constant.
struct FrameParams {
  uint32_t step, seed_lo, seed_hi, frame;
  double k0;
};

// One scene of a multi-scene batch as its chains see it: their index range,
// path length L and PSS dimension d, the scene's first pixel in the shared
// accumulation image, its k0 and its tour counter.  Device memory, so a
// replayed graph picks up k0 estimated after capture.
struct SceneChains {
  unsigned long long chain0, n;
  int L, d;
  uint32_t pix0, pad;
  double k0;
  unsigned long long* tour_count;
};

struct StepArgs {
  DevScene S;
  // multi-scene batch (null: the single scene S): per-scene BVH and camera,
  // per-scene chain table, and the scene of every chain
  const DevScene* scenes;
  const SceneChains* sc;
  const uint8_t* chain_scene;
  DevMixture M;
  int target;  // 0 scene, 1 mixture
  float* x;          // [d][N]
  float* score;      // [d][N]
  float* xp;         // [d][N] MALA: the proposal
  float* sp;         // [d][N] MALA: the score at the proposal
  float4* cur;       // [N] MALA: f (rgb) and pixel of the current state
  uint8_t* killed;   // [N]
  float* logp;       // [N]
  SplatRec* rec;     // [N] slice for this step (null: no records)
  unsigned long long N;
  int d, L;
  uint32_t step;
  const FrameParams* fp;  // non-null: step, RNG key and k0 from device memory (graph replay)
  Rng rng;
  float stddev, gamma_tilde, h, eps;
  double k0;
  int rb, drift, init;
  int estimate_only;  // init pass that only sums p (k0 unknown yet)
  const uint2* order;  // [N] (key, chain) pairs: thread t works on chain order[t].y; null = identity
  uint8_t* plen;       // [N] path length of the chain's last evaluation (null: not recorded)
  unsigned long long* tour_count;
  unsigned long long* rays;
  unsigned long long* node_visits;  // stats mode only
  unsigned long long* tri_tests;    // stats mode only
  double* p_partial;  // [gridDim.x] init only
  uint32_t* err;
  int refill;  // persistent traversal: refill a warp below this many busy lanes
  int conductors;  // some material is a conductor: the shading passes that handle them run
  int bvh8;        // the persistent passes walk the 8-wide BVH (every scene has one)
  int two_level;   // the persistent passes walk the two-level BVH of an instanced scene
  // camera-ray order (null: chain order): wf_begin writes (key, chain) with
  // key = the pixel's Morton code (above it the scene of a batch chain)
  uint2* ray_keys;
  int key_shift;  // Morton bits: a batch chain's key is (scene << key_shift) | morton
};

// (key, chain) pairs for the work order of the next step
void launch_order_keys(const uint8_t* killed, const uint8_t* plen, unsigned long long N, uint2* keys,
                       cudaStream_t s);

// ---------------------------------------------------------------- wavefront
// NEE shadow ray of one vertex: origin + tmax, direction + chain id bits,
// pending contribution + excluded triangle, second excluded triangle.
struct __align__(16) ShadowRec {
  float4 o_tmax, wi_chain, contrib_ex;
  int ex1, pad0, pad1, pad2;
};
// counters: [k] = rays of bounce k (1..16), [17 + k] = shadow rays of bounce
// k (1..16), [34 + k] = fetch position of the traversal pass of bounce k
// (1..17; k = 0: the tail pass), [52 + s] = surviving chains with s path
// segments (0..16), queued for the adjoint
constexpr int kWfShadowCount0 = 17;
constexpr int kWfFetch0 = 34;
constexpr int kWfAdjBucket0 = 52;
constexpr int kWfCounts = 69;
static_assert(kWfFetch0 + kMaxPathLen + 1 < kWfAdjBucket0, "fetch counters overlap the adjoint buckets");
static_assert(kWfShadowCount0 + kMaxPathLen < kWfFetch0, "shadow counts overlap the fetch counters");
static_assert(kWfAdjBucket0 + kMaxPathLen < kWfCounts, "adjoint buckets exceed the counter block");
struct WfBuffers {
  float4* slot;        // [N][4] path state
  int* hit;            // [N] closest-hit triangle of the current ray
  uint32_t* queue[2];  // ray queues (ping-pong), chain ids
  ShadowRec* shadow;   // [N] shadow queue of the current bounce
  uint32_t* adj;       // [17][N] chains for the adjoint pass, by path length
  uint32_t* counts;    // [kWfCounts]
  float4* tape;        // [L][3][N]
};
size_t wf_bytes(unsigned long long N, int L);
WfBuffers wf_carve(void* base, unsigned long long N, int L);

// Phases timed by the optional profiler (events recorded around launches).
enum Phase { kPhBegin = 0, kPhTrace, kPhShade, kPhShadow, kPhFinish, kPhAdjoint, kPhFused, kPhFd, kPhSplat,
             kPhOrder, kPhTail, kPhCount };
struct PhaseHook {
  void (*mark)(void* user, int phase, bool begin, int bounce);
  void* user;
  // bounce: 1..L for the per-bounce passes, 0 otherwise
  void operator()(int phase, bool begin, int bounce = 0) const {
    if (mark) mark(user, phase, begin, bounce);
  }
};

// One adjoint-drift Restore step on a scene, bounce by bounce; returns the
// number of kernels (and memsets) issued.  Modes: kWfStep (the step), and
// the two halves of a single-pass initialisation whose k0 is estimated from
// the same evaluation: kWfInitEval (Init's evaluation; p of every chain to
// p_out, the adjoint for every chain, no clock) then kWfInitClock (the
// kill clock and records from the stored path results, once k0 is known).
enum WfMode { kWfStep = 0, kWfInitEval = 1, kWfInitClock = 2 };
// Launch shape of the persistent traversal pass: blocks per SM (0: as many
// as stay resident) and the lane count below which a warp refills.
struct WfTuning {
  int blocks_per_sm = 0;
  int refill = 16;
  int tail_bounce = 0;  // 0: every bounce as its own passes; k >= 1: one persistent pass from shading bounce k on
};
// Sorting of the camera rays by pixel before the first traversal: the key
// buffer (a.ray_keys), its ping-pong partner, the sort scratch and the
// number of key bits.  keys == null: rays in chain order.
struct RayOrder {
  uint2* keys = nullptr;
  uint2* alt = nullptr;
  void* scratch = nullptr;
  int bits = 0;
};
int launch_wavefront_step(const StepArgs& a, const WfBuffers& w, bool stats, int n_sm, const WfTuning& tune,
                          const PhaseHook& hook, cudaStream_t s, WfMode mode = kWfStep, float* p_out = nullptr,
                          const RayOrder& order = RayOrder{});
// step index += 1 on the device (graph replay)
void launch_advance_step(uint32_t* step, cudaStream_t s);

int step_block_size();
size_t step_smem_bytes();
void launch_step(const StepArgs& a, bool stats, cudaStream_t s);

struct FdArgs {
  DevScene S;
  DevMixture M;
  int target;
  const float* x;
  float* score;
  const uint8_t* killed;
  unsigned long long N;
  int d, L;
  float eps, fd_h;
  unsigned long long* rays;
  uint32_t* err;
};
void launch_fd_score(const FdArgs& a, cudaStream_t s);

struct EvalArgs {
  DevScene S;
  DevMixture M;
  int target;
  const float* x;  // [M][d]
  float* logp;     // [M]
  float* grad;     // [M][d] or null
  int* pix;        // [M] or null
  float* f;        // [M][3] or null
  long long Mpts;
  int d, L;
  float eps;
  uint32_t* err;
};
void launch_eval(const EvalArgs& a, cudaStream_t s);

// L* p / p at query points of a 2-D mixture target (dr_bias.cu)
struct LstarArgs {
  DevMixture M;
  const float* y;  // [n_pts][2]
  long long n_pts;
  double stddev, h, gamma_tilde, eps, radius;
  int n;          // quadrature nodes per side
  double* out;    // [n_pts]
};
void launch_lstar(const LstarArgs& a, cudaStream_t s);

void launch_trace(const DevScene& S, const float* rays, long long n, int exclude, int* tri, float* t, uint32_t* err,
                  cudaStream_t s);
// launch_trace with each ray's node steps and triangle tests counted
void launch_trace_stats(const DevScene& S, const float* rays, long long n, int exclude, int* tri, float* t,
                        uint32_t* nodes, uint32_t* tests, uint32_t* err, cudaStream_t s);
void launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, long long n, cudaStream_t s);
void launch_sum_doubles(const double* in, int n, double* out, cudaStream_t s);
// partial[b] = FP64 sum of p over the fused step kernel's block b, in its order
void launch_block_sums(const float* p, unsigned long long N, double* partial, cudaStream_t s);
// Stratified path tracing of the same f: part [n_chunks][W*H][3] FP64
// scratch, mean [W*H][3] = per-pixel mean of f / (W H) over spp samples.
void launch_pt(const DevScene& S, int L, uint32_t spp, int n_chunks, Rng rng, double* part, double* mean,
               unsigned long long* rays, uint32_t* err, cudaStream_t s);

}  // namespace dr
