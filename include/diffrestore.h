/* diffrestore.h — C ABI of libdiffrestore (GB300, sm_103a).
 *
 * The data-parallel hot path of Diffusion Restore (arxiv 2605.08916): many
 * independent Jump Restore chains ("tours") in primary sample space, each
 * step evaluating the path contribution f(x), p(x) = lum(f) + eps and
 * grad log p, taking one Euler-Maruyama step of the nonreversible Langevin
 * local dynamics, running the hold/kill clock, regenerating killed chains
 * from the uniform distribution, and splatting dt * f / p into an FP64 image.
 *
 * Conventions for every entry point:
 *  - Return value: DR_OK (0) or a negative DR_ERR_* code; dr_last_error()
 *    gives a thread-local message for the most recent failure.  No call
 *    aborts, throws or traps.
 *  - The library owns all device memory it allocates; buffers passed in are
 *    only read (or written where stated) during the call or, for device
 *    pointers, in stream order on the context's stream.
 *  - "host" pointers are read / written synchronously; "device" pointers must
 *    point to memory of the context's device.
 *  - Work is issued on the CUDA stream given to dr_create (0 = legacy
 *    default stream) and is stream-ordered unless a call says it synchronises.
 *  - Array layouts are row-major and tightly packed.
 */
#ifndef DIFFRESTORE_H_
#define DIFFRESTORE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DR_OK = 0,
  DR_ERR_INVALID_ARG = -1,   /* bad pointer, size or value */
  DR_ERR_STATE = -2,         /* call out of order (e.g. step before init) or empty estimate */
  DR_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  DR_ERR_OOM = -4,           /* device allocation failed */
  DR_ERR_DEVICE_CHECK = -5,  /* a kernel reported a checked condition (stack overflow, non-finite value) */
  DR_ERR_TIMEOUT = -6        /* a bounded device wait gave up */
};

enum { DR_DRIFT_NONE = 0, DR_DRIFT_FD = 1, DR_DRIFT_ADJOINT = 2, DR_DRIFT_MALA = 3 };

enum { DR_MAX_PATH_LEN = 16 }; /* L <= 16, so d = 2 + 4 (L - 1) <= 62 */

typedef struct dr_ctx dr_ctx;

/* Parameters of the Diffusion Restore process (Def. 2, Sec. 5.3; Sec. 6
 * "Parameter choices").
 *   max_path_len    L, number of path segments from the camera (1..16);
 *                   the PSS dimension is d = 2 + 4 (L - 1).
 *   drift_mode      DR_DRIFT_NONE (score 0), DR_DRIFT_FD (central finite
 *                   differences of log p with step fd_h), DR_DRIFT_ADJOINT
 *                   (hand-written reverse-mode gradient of log p), or
 *                   DR_DRIFT_MALA: MALA Restore, the comparison method of
 *                   Sec. 6 (Jump Restore whose local move is a
 *                   Metropolis-adjusted Langevin step: proposal
 *                   x + (stddev^2 / 2) grad log p(x) + stddev xi with the
 *                   normals of Alg. 4 and no rotation, accepted with the
 *                   Metropolis-Hastings probability in FP64, torus
 *                   differences to the nearest image; the paper runs it with
 *                   holding rate 1, i.e. dt = 1).  MALA runs in the fused
 *                   execution (one thread per chain-step), on a scene or a
 *                   mixture, not in a batch; its chains cannot be
 *                   checkpointed (dr_state_save gives STATE).
 *   rb_weight       0: the paper's exponential race of Alg. 1 (hold time
 *                   ~ Exp(h), kill time ~ Exp(k), splat weight = the smaller);
 *                   1: its Rao-Blackwellisation (weight 1 / (h + k), killed
 *                   with probability k / (h + k)).
 *   steps_per_splat records buffered before an automatic splat (>= 1).
 *   stddev          sqrt(dt) * sigma, the per-step noise scale (paper: 5e-3).
 *   dt              Euler-Maruyama step; holding rate h = 1 / dt (paper 1e-5).
 *   gamma_tilde     dt * gamma / 2, the rotation scale of Alg. 4.
 *   eps             density floor, p = lum(f) + eps (paper 1e-8).
 *   fd_h            finite-difference step for DR_DRIFT_FD.
 *   m               mean tour length target in k0 = p_lambda / (m dt)
 *                   (Eq. killing-rate-constant; paper m = 64).
 *   k0              killing constant; if <= 0, dr_chains_init estimates
 *                   p_lambda as the mean of p over the initial uniform
 *                   samples and sets k0 = p_lambda / (m dt). */
typedef struct {
  int32_t max_path_len;
  int32_t drift_mode;
  int32_t rb_weight;
  int32_t steps_per_splat;
  float stddev;
  float dt;
  float gamma_tilde;
  float eps;
  float fd_h;
  float m;
  double k0;
} dr_params;

/* Library version (major * 10000 + minor * 100 + patch). */
int dr_version(void);

/* Message for the most recent failing call on this thread ("" if none).
 * The returned pointer stays valid until the thread's next failing call. */
const char* dr_last_error(void);

/* Creates a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  *out receives
 * the handle.  Errors: INVALID_ARG (out NULL, bad device), CUDA. */
int dr_create(dr_ctx** out, int device, void* cuda_stream);

/* Synchronises the context's stream and frees everything it owns. NULL is OK. */
int dr_destroy(dr_ctx* ctx);

/* Uploads a triangle scene and builds its BVH on the device (Sec. 4.3: the
 * scene the tours trace; a change invalidates the chains, which must be
 * re-initialised).  All pointers are HOST pointers, copied before return.
 *   verts      float [nv * 3] vertex positions
 *   tris       int32 [nt * 3] vertex indices (counter-clockwise = front)
 *   normals    float [nv * 3] per-vertex shading normals, or NULL (flat);
 *              a triangle is smooth-shaded only if its three vertex
 *              normals are all non-zero (zero rows mark flat meshes)
 *   tri_mat    int32 [nt] material index per triangle
 *   mats       float [nm * 12] materials: type (0 diffuse, 1 glossy GGX coat
 *              over Lambertian, 2 smooth dielectric, 3 black emitter,
 *              4 rough GGX conductor), albedo rgb, roughness, ior, emission
 *              rgb, f0, 0, 0.  A conductor (pbrt's conductor, Sec. 6 "Test
 *              scenes") stores the real part eta of its complex index of
 *              refraction (rgb, > 0) in the albedo slots and the imaginary
 *              part k (rgb, > 0) in the last three slots.  Emission
 *              is one-sided along cross(v1 - v0, v2 - v0); emitting
 *              triangles form the light set used by next-event estimation.
 *   camera     float [10]: eye xyz, look-at xyz, up xyz, vertical fov (deg)
 *   width, height  image size in pixels (>= 1; width * height < 2^31)
 * Synchronises the stream.  Errors: INVALID_ARG, OOM, CUDA, DEVICE_CHECK.
 * INVALID_ARG leaves the context as it was; after any other error it has no
 * scene (and no chains) until an upload succeeds. */
int dr_scene_upload(dr_ctx* ctx, const float* verts, int32_t nv, const int32_t* tris, const float* normals,
                    int32_t nt, const int32_t* tri_mat, const float* mats, int32_t nm, const float* camera,
                    int32_t width, int32_t height);

/* One scene of a multi-scene batch: the arrays and meaning of
 * dr_scene_upload (HOST pointers, copied), plus the scene's own path length
 * (1..16) and number of chains. */
typedef struct {
  const float* verts;
  int32_t nv;
  const int32_t* tris;
  const float* normals;
  int32_t nt;
  const int32_t* tri_mat;
  const float* mats;
  int32_t nm;
  const float* camera;
  int32_t width, height;
  int32_t max_path_len;
  uint64_t n_chains;
} dr_scene_desc;

/* Uploads n_scenes (1..255) scenes as one batch (a workload of many views
 * of uneven size and path length advanced together).  Each scene gets its
 * own BVH (binary and 4-wide; every scene needs >= 2 triangles), camera,
 * image, k0 and tourCount; their chains are laid out scene after scene in
 * one state array (PSS dimension of the longest path), and every step of
 * all scenes runs in one sequence of bounce-by-bounce launches whose ray
 * queues mix the scenes.  Chain j of scene s draws from the Philox stream
 * with key (seed_lo, seed_hi + s) and chain word j - (first chain of s), so
 * a scene evolves exactly as it would in a context of its own with that
 * key.  The images share one FP64 accumulator, scene after scene.  Then
 * dr_chains_init (n_chains = the sum over scenes, prm->drift_mode must be
 * DR_DRIFT_ADJOINT; prm->max_path_len is ignored), dr_step / dr_frame /
 * dr_splat as usual, and dr_resolve_scene per scene.  Synchronises.
 * Errors: INVALID_ARG, OOM, CUDA, DEVICE_CHECK. */
int dr_scenes_upload_batch(dr_ctx* ctx, const dr_scene_desc* scenes, int32_t n_scenes);

/* A mesh of an instanced scene (object space; HOST pointers, copied):
 * verts float [nv * 3], tris int32 [nt * 3] (counter-clockwise = front),
 * normals float [nv * 3] per vertex or NULL (flat), tri_mat int32 [nt]. */
typedef struct {
  const float* verts;
  int32_t nv;
  const int32_t* tris;
  int32_t nt;
  const float* normals;
  const int32_t* tri_mat;
} dr_mesh_desc;

/* One placement of a mesh: xform is the object-to-world affine map,
 * row-major 3 x 4 (world = A p + t with rows (A_r0, A_r1, A_r2, t_r)), A
 * invertible; material >= 0 replaces the mesh's per-triangle materials, -1
 * keeps them. */
typedef struct {
  int32_t mesh;
  int32_t material;
  float xform[12];
} dr_instance_desc;

/* Uploads an instanced scene (Sec. 6 "Test scenes": objects placed in a
 * scene; the two-level acceleration structure of RT pipelines, Sec. 4.3).
 * The scene is by definition its flattening: instance after instance, each
 * mesh vertex p goes to world position ((A_r0 p.x + A_r1 p.y) + A_r2 p.z) +
 * t_r per row r in FP64, rounded to float; normals go through the inverse
 * transpose (the inverse by cofactors over the determinant, in FP64);
 * triangle ids are the flattened order (instance-major); a mesh without
 * normals is flat-shaded.  Everything dr_scene_upload builds is built for
 * the flattened scene; in addition, when DR_OPT_TWO_LEVEL is 1 at the
 * upload and there are at least 2 instances, a two-level BVH: a 4-wide BLAS
 * per mesh (object space, the context's builder) and a 4-wide TLAS over the
 * instances' world boxes with one instance per leaf, which the
 * bounce-by-bounce passes then walk, rays mapped into each instance's object
 * space (see dr_two_level_info).
 * Other arguments as in dr_scene_upload.  Synchronises.
 * Errors: INVALID_ARG (bad index, singular or non-finite transform, sizes),
 * OOM, CUDA, DEVICE_CHECK. */
int dr_scene_upload_instanced(dr_ctx* ctx, const dr_mesh_desc* meshes, int32_t n_meshes,
                              const dr_instance_desc* instances, int32_t n_instances, const float* mats, int32_t nm,
                              const float* camera, int32_t width, int32_t height);

/* The two-level BVH of an instanced scene: instances, TLAS nodes and the
 * BLASes' total nodes (HOST outputs, each may be NULL).  Errors: STATE (no
 * instanced scene, fewer than 2 instances, or one whose two-level walk
 * could need more stack than the kernels hold). */
int dr_two_level_info(dr_ctx* ctx, int32_t* n_instances, int32_t* n_tlas_nodes, int32_t* n_blas_nodes);

/* Resolve (Alg. 3) of scene `scene` of a batch into the FP32 DEVICE buffer
 * out_rgb [W_s * H_s * 3] with that scene's k0 and tourCount.  Errors as
 * dr_resolve, plus STATE when no batch is uploaded, INVALID_ARG for a bad
 * scene index. */
int dr_resolve_scene(dr_ctx* ctx, int32_t scene, float* out_rgb);

/* Per-scene counters of a batch (HOST outputs, may be NULL): completed
 * tours and k0.  Synchronises. */
int dr_get_scene_counters(dr_ctx* ctx, int32_t scene, uint64_t* tour_count, double* k0);

/* Uses an analytic target instead of a scene: an isotropic Gaussian mixture
 * on the torus T^d, p = g + eps with g(x) = sum_k w[k] N(x; mu[k],
 * sig[k]^2 I) (differences to the nearest image), or the constant `cval`
 * when K = 0.  f = (g, g, g); the pixel comes from (x0, x1) on a
 * width x height grid.  HOST pointers w [K], mu [K * d], sig [K].
 * d must be even, 2..62.  Errors: INVALID_ARG, OOM, CUDA.  INVALID_ARG
 * leaves the context as it was; after any other error it has no target. */
int dr_target_mixture(dr_ctx* ctx, int32_t d, int32_t K, const float* w, const float* mu, const float* sig,
                      float cval, int32_t width, int32_t height);

/* Initialize (Alg. 1) for n_chains chains: each chain j draws x ~ U(T^d)
 * from its Philox4x32-10 stream (key = seed, counter = (step, j, block,
 * frame << 4 | purpose)), evaluates f and p, runs the clock and records its
 * splat.  Clears the image accumulator and tourCount.  If prm->k0 <= 0,
 * k0 = p_lambda / (m dt) with p_lambda estimated from the same initial
 * samples (Eq. killing-rate-constant), computed before the init clock runs.
 * prm is a HOST pointer, copied.  Synchronises when k0 is estimated.
 * Errors: STATE (no scene/target), INVALID_ARG, OOM, CUDA, DEVICE_CHECK.
 * INVALID_ARG leaves earlier chains in place; after any other error the
 * context has no chains (dr_step and the other chain calls give STATE)
 * until an init succeeds. */
int dr_chains_init(dr_ctx* ctx, uint64_t n_chains, uint64_t seed, uint32_t frame, const dr_params* prm);

/* Evolve (Alg. 2 with LocalDynamics, Alg. 4) n_steps times: killed chains
 * regenerate from U(T^d), the others move with the drift of the score
 * stored at their current point; then each chain accumulates at its new
 * point.  Records are splatted automatically when the buffer of
 * steps_per_splat steps is full (before the step that would overflow it),
 * so after the call the last step's records are still readable.
 * Asynchronous.  Errors: STATE, CUDA. */
int dr_step(dr_ctx* ctx, uint32_t n_steps);

/* Splats all buffered records into the FP64 accumulator (the accumulation
 * of Alg. 1, without atomics, deterministic).  Asynchronous. */
int dr_splat(dr_ctx* ctx);

/* Resolve (Alg. 3): out_rgb[i] = k0 / tourCount * accum[i] for the W*H*3
 * FP32 DEVICE buffer out_rgb (row-major pixels, row 0 at the top, RGB).
 * Splats pending records first.  Zero image when tourCount = 0, and then
 * returns DR_ERR_STATE (checked with a synchronisation unless the stream is
 * being captured). */
int dr_resolve(dr_ctx* ctx, float* out_rgb);

/* Copies the chain state to HOST buffers (any may be NULL): x and score
 * [N * d] row-major per chain (score = grad log p at x, valid for chains
 * that are not killed), killed [N], logp [N] of the last step, pix [N] and
 * val [N * 3] (the last step's splat record).  Synchronises. */
int dr_readback_state(dr_ctx* ctx, float* x, float* score, uint8_t* killed, float* logp, int32_t* pix, float* val);

/* Copies the FP64 accumulator (W * H * 3, after splatting pending records)
 * into a HOST buffer.  Synchronises. */
int dr_readback_accum(dr_ctx* ctx, double* accum);

/* Counters (HOST outputs, any may be NULL): completed tours (tourCount of
 * Sec. 4.3), k0 in use, steps taken since init (init = step 0), rays traced
 * since init, and the estimated p_lambda (0 if k0 was given).  Synchronises. */
int dr_get_counters(dr_ctx* ctx, uint64_t* tour_count, double* k0, uint64_t* steps, uint64_t* rays,
                    double* p_lambda);

/* Batched evaluation at M points, DEVICE buffers: x [M * d] row-major,
 * logp [M] = log(lum f + eps), grad [M * d] = grad log p (hand-written
 * adjoint, or NULL), pix [M] or NULL, f [M * 3] or NULL.  Uses the uploaded
 * scene (L from max_path_len) or mixture target.  Asynchronous. */
int dr_eval_logp(dr_ctx* ctx, int32_t max_path_len, const float* x, int64_t M, float* logp, float* grad,
                 int32_t* pix, float* f);

/* The bias term of the modified killing rate (Sec. 5.2, Eq. bias and
 * Eq. adjoint-bias; the diagnostic of App. C): (L* p / p)(y) =
 * h ((K* p)(y) / p(y) - 1) for the mixture target on T^2 (dr_target_mixture
 * with d = 2), where K is the Euler-Maruyama kernel of Alg. 4 with the
 * stddev and gamma_tilde of prm, h = 1 / prm->dt, p = g + prm->eps, and
 * (K* p)(y) = int p(x) K(x, y) dx by the trapezoid rule in FP64 over the
 * square of half-width radius * stddev around y with n x n nodes (kernel
 * differences to the nearest torus image).  With the modified killing rate
 * the Restore estimate is biased by -(L* p / p).
 *   prm   HOST, only stddev, dt, gamma_tilde and eps are read.
 *   y     DEVICE float [M * 2] query points; out DEVICE double [M].
 *   n     2..4097 nodes per side (e.g. 129 with radius 8: spacing
 *         stddev / 8).
 * Asynchronous.  Errors: INVALID_ARG, STATE (no 2-D mixture target), CUDA. */
int dr_lstar_over_p(dr_ctx* ctx, const dr_params* prm, const float* y, int64_t M, float radius, int32_t n,
                    double* out);

/* Closest-hit queries through the BVH: rays [n * 6] (origin, direction;
 * DEVICE), tri [n] original triangle id or -1, t [n] distance (inf on miss).
 * `exclude` is a triangle id to skip (-1: none).  Asynchronous.
 * Errors: INVALID_ARG (NULL pointer, n < 0), STATE (no single scene), CUDA. */
int dr_trace_closest(dr_ctx* ctx, const float* rays, int64_t n, int32_t exclude, int32_t* tri, float* t);

/* dr_trace_closest with each ray's walk counted: node_steps [n] the inner
 * nodes the walk visited and tri_tests [n] the triangles it tested (DEVICE
 * uint32), the per-ray terms of the traversal statistics that give the
 * roofline's algorithmic bytes (112 B per 4-wide node visit, 48 B per
 * triangle test).  The walk is the one the persistent passes take (the
 * 4-wide BVH when built).  Asynchronous.
 * Errors: INVALID_ARG, STATE (no single scene), CUDA. */
int dr_trace_closest_counted(dr_ctx* ctx, const float* rays, int64_t n, int32_t exclude, int32_t* tri, float* t,
                             uint32_t* node_steps, uint32_t* tri_tests);

/* Philox4x32-10 (Salmon et al. 2011, cited in Sec. 4.3) on DEVICE buffers:
 * ctr [n * 4], key [n * 2] -> out [n * 4].  cuda_stream may be NULL.
 * Asynchronous. */
int dr_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* cuda_stream);

/* Splats M caller-made records (DEVICE, 16 bytes each: uint32 pixel index,
 * float r, g, b) into the accumulator with the same sort + reduce as the
 * chain records.  Pixel indices must be < W * H: a record at or above it
 * is not added, and the call returns DEVICE_CHECK.  The other pixels'
 * sums are then unspecified (the sort orders by the low key bits only), so
 * clear the image with dr_clear_image.  The context's own device-check state
 * is not touched.  Allocates temporary device memory and synchronises.
 * Errors: INVALID_ARG, STATE (no image yet), OOM, CUDA, DEVICE_CHECK. */
int dr_splat_records(dr_ctx* ctx, const void* recs, int64_t M);

/* Resets the accumulator and tourCount without touching the chains (a new
 * accumulation window over the same tours).  Asynchronous. */
int dr_clear_image(dr_ctx* ctx);

/* Checkpoint: serialises the chain state, counters, k0 and the FP64
 * accumulator into a HOST buffer.  With host_buf NULL, *bytes receives the
 * size needed.  A run resumed with dr_state_load continues bit-for-bit like
 * an uninterrupted one (the RNG is counter-based).  Synchronises.
 * dr_state_load reads `bytes` bytes of host_buf and checks them before any
 * device work: a buffer that is not a checkpoint of this version, is
 * truncated, was saved for another image or dimension, or holds a chain
 * count outside [1, 2^31], invalid parameters or a k0 that is not positive
 * and finite gives INVALID_ARG (the context is left as it was).
 * Errors: INVALID_ARG (also NULL arguments), STATE (save: no chains; load:
 * no target uploaded; either: a batch context), OOM, CUDA. */
int dr_state_save(dr_ctx* ctx, void* host_buf, size_t* bytes);
int dr_state_load(dr_ctx* ctx, const void* host_buf, size_t bytes);

/* Traversal statistics mode: when enabled, steps also count BVH node
 * visits and triangle tests (a separate kernel instantiation; the default
 * kernels carry no counters).  dr_get_traversal_stats returns the totals
 * since the last enable. */
int dr_set_stats(dr_ctx* ctx, int enable);
int dr_get_traversal_stats(dr_ctx* ctx, uint64_t* node_visits, uint64_t* tri_tests, uint64_t* rays);

/* BVH summary: number of inner nodes, triangles, maximum depth (root = 1).
 * Synchronises. */
int dr_bvh_info(dr_ctx* ctx, int32_t* n_nodes, int32_t* n_tris, int32_t* max_depth);

/* The 4-wide BVH that dr_scene_upload collapses from the binary one on the
 * host (a subtree of at most 4 triangles becomes a leaf where the surface-
 * area heuristic favours it; each inner node takes up to 4 children by
 * opening its largest inner grandchildren).  Node: 112 B = lo.x[4], hi.x[4],
 * lo.y[4], hi.y[4], lo.z[4], hi.z[4], links[4].  HOST outputs (each may be
 * NULL): node count, depth (root = 1), and the most traversal-stack entries
 * a traversal can hold.  Errors: STATE (no scene, or none was built: a
 * one-triangle scene, or a tree whose traversal would need more stack than
 * the kernels hold; rays then use the binary BVH). */
int dr_bvh4_info(dr_ctx* ctx, int32_t* n_nodes, int32_t* max_depth, int32_t* stack_need);

/* Copies the 4-wide BVH to HOST buffers, for tools that walk it on the
 * host.  nodes [n_nodes * 28] floats (dr_bvh4_info's count): per node the
 * children's box planes as six groups of four (lo x, hi x, lo y, hi y,
 * lo z, hi z; slot k in entry k of each group), then four int32 links: an
 * inner child's node index (>= 0), a leaf (bit 31 set; first triangle =
 * (link & 0x7fffffff) >> 3, count = (link & 7) + 1), or 0x7fffffff (empty;
 * an empty slot's box is inverted, lo = +inf and hi = -inf, so that every
 * slab test misses it).
 * tris [n_tris * 12] floats: per triangle in leaf order v0 and the int32
 * original id, e1 = v1 - v0 and 0, e2 = v2 - v0 and 0.  Synchronises.
 * Errors: INVALID_ARG, STATE (no single scene or no 4-wide BVH), CUDA. */
int dr_bvh4_download(dr_ctx* ctx, float* nodes, float* tris);

/* Quality of the 4-wide BVH by the surface-area heuristic (the measure its
 * leaf decision minimises): for a ray that hits the root box, with each
 * box entered with probability area(box) / area(root box), the expected
 * number of node steps (the root's included; HOST output node_steps) and
 * of triangle tests (HOST output tri_tests).  Computed at upload.  Each
 * output may be NULL.  Errors: STATE (no 4-wide BVH). */
int dr_bvh4_sah(dr_ctx* ctx, double* node_steps, double* tri_tests);

/* The 8-wide compressed BVH of the uploaded scene, built at upload when
 * DR_OPT_BVH_WIDTH is 8: the binary tree collapsed with the same leaf rule
 * into nodes of up to 8 children, numbered breadth first (a node's inner
 * children consecutive, its leaf triangles consecutive).  Node: 80 B = the
 * node box origin (3 floats), three signed 8-bit exponents and the
 * inner-child mask, the first inner child and first triangle, 8 leaf
 * descriptors, and per child and plane an 8-bit offset (the child box is
 * widened to the 8-bit grid, never narrowed).  Children take slots by the
 * ray-octant heuristic (a ray visits slot k ^ octant k-th).  HOST outputs
 * (each may be NULL): node count and depth (root = 1).  Errors: STATE (no
 * scene, or none was built: width 8 not set before the upload, fewer than
 * 2 triangles, or a tree deeper than the traversal stack holds). */
int dr_bvh8_info(dr_ctx* ctx, int32_t* n_nodes, int32_t* max_depth);

/* Number of kernels this context has launched since creation (a host-side
 * count kept at every launch site; HOST output). */
int dr_get_launch_count(dr_ctx* ctx, uint64_t* launches);

/* Ordinary Monte Carlo (path tracing, the paper's PT method, Sec. 6) over
 * the same f: per pixel, spp samples with the film pair stratified to the
 * pixel and the other coordinates uniform from Philox (key = seed, counter
 * = (sample, pixel, block, 3)).  out_mean: DEVICE FP64 [W * H * 3], the
 * per-pixel mean of f / (W H), i.e. the pixel radiance estimate in the same
 * units as dr_resolve.  Allocates temporary device memory; synchronises.
 * Errors: STATE (no scene), INVALID_ARG, OOM, CUDA, DEVICE_CHECK. */
int dr_pt_render(dr_ctx* ctx, int32_t max_path_len, uint32_t spp, uint64_t seed, double* out_mean);

/* Execution options.  They change speed, not the method: results are the
 * same up to floating-point contraction order (DR_OPT_WAVEFRONT) and the
 * triangle picked on a shared edge (DR_OPT_TWO_LEVEL), as stated below.
 *   DR_OPT_WAVEFRONT   1: adjoint-drift (or no-drift) steps on a scene
 *                      run bounce by bounce over compacted queues of live
 *                      paths (trace / shade / shadow kernels per bounce,
 *                      the per-segment tape in device memory, the adjoint
 *                      pass over surviving chains only, skipped without a
 *                      drift); 0: one fused kernel, one
 *                      thread per chain-step; -1 (default): wavefront from
 *                      2^17 chains up, fused below.  The two agree to
 *                      floating-point contraction order (last-bit level).
 *   DR_OPT_WORK_ORDER  for the fused kernel only: 1 orders chains by
 *                      (killed last step, previous path length) with one
 *                      stable radix pass before each step so that warps
 *                      trace paths of similar cost; 0 (default): chain order.
 *   DR_OPT_PROFILE     1: record CUDA events around each pass of dr_step /
 *                      dr_splat (not inside dr_frame graphs) and accumulate
 *                      their durations per phase (see dr_get_profile).
 *   DR_OPT_TRAVERSE_BLOCKS  blocks per SM of the persistent traversal pass
 *                      (1..64, capped at the resident count; 0 (default):
 *                      all resident blocks).
 *   DR_OPT_REFILL      a traversal warp fetches new rays once fewer than
 *                      this many of its 32 lanes are busy (1..32; default 16).
 *   DR_OPT_RAY_ORDER   1: before the first traversal of a bounce-by-bounce
 *                      step the camera rays are sorted by pixel (Morton
 *                      order; scene first in a batch), so that neighbouring
 *                      lanes trace neighbouring rays; 0: chain order; -1
 *                      (default): on from 2^17 triangles (a batch counts
 *                      all its scenes).  Results are the same either way.
 *   DR_OPT_TAIL_BOUNCE k >= 1: from the shading of bounce k on, each path
 *                      runs to its end inside one persistent pass (its
 *                      shadow rays, next rays and shading interleaved per
 *                      lane) instead of one launch per pass and bounce; the
 *                      arithmetic per path is the same.  0: no tail pass;
 *                      -1 (default): automatic.  Bounce-by-bounce passes
 *                      over a 4-wide, 8-wide or two-level BVH.
 *   DR_OPT_BVH_WIDTH   4: rays traverse the 4-wide BVH collapsed from the
 *                      binary one at scene upload (when it was built, see
 *                      dr_bvh4_info); 2: the binary BVH; 0 (default): the
 *                      4-wide one; 8: set before dr_scene_upload (or the
 *                      batch upload), also builds the 8-wide compressed BVH
 *                      (dr_bvh8_info), which the bounce-by-bounce passes
 *                      then walk (the fused kernel keeps the 4-wide one).
 *                      All return the same closest hit (ties: smaller id).
 *   DR_OPT_TWO_LEVEL   1 (set before dr_scene_upload_instanced): an
 *                      instanced scene also gets a two-level BVH, which the
 *                      bounce-by-bounce passes walk; 0 (default, or set to
 *                      0 later): they walk the flattened scene's BVH (faster
 *                      here: the object-space maps cost more than the
 *                      shallower trees save).  The two test triangles in
 *                      object vs world space, so a hit on an edge shared by
 *                      two triangles can go to either (the hit point and
 *                      shading always come from the flattened triangle).
 * Errors: INVALID_ARG (unknown option or value). */
enum { DR_OPT_WORK_ORDER = 1, DR_OPT_WAVEFRONT = 2, DR_OPT_PROFILE = 3, DR_OPT_BVH_WIDTH = 4,
       DR_OPT_TRAVERSE_BLOCKS = 5, DR_OPT_REFILL = 6, DR_OPT_RAY_ORDER = 7, DR_OPT_TAIL_BOUNCE = 8,
       DR_OPT_TWO_LEVEL = 9 };
int dr_set_option(dr_ctx* ctx, int32_t option, int32_t value);

/* Per-phase device time accumulated since the last call while DR_OPT_PROFILE
 * is on (synchronises, then resets the totals).  HOST outputs ms[i] and
 * counts[i] (launches timed; may be NULL) for i < n, phases in order:
 * 0 wavefront begin (Evolve + camera rays), 1 closest-hit traversal,
 * 2 shading / NEE / BSDF sampling, 3 shadow-ray traversal, 4 clock and
 * records, 5 adjoint, 6 fused step kernel, 7 finite-difference score,
 * 8 splat (sort + reduce), 9 work-order / camera-ray sort, 10 the tail
 * pass (shading and traversal of the late bounces, DR_OPT_TAIL_BOUNCE). */
enum { DR_PHASES = 11 };
int dr_get_profile(dr_ctx* ctx, double* ms, uint64_t* counts, int32_t n);

/* The bounce-by-bounce part of the same profile: HOST output ms[3 *
 * n_bounces], rows closest-hit traversal, shading, shadow-ray traversal,
 * column k - 1 = bounce k, accumulated since the last dr_get_profile (which
 * also clears these; this call clears nothing).  Synchronises.
 * Errors: INVALID_ARG (n_bounces outside 1..16). */
int dr_get_bounce_profile(dr_ctx* ctx, double* ms, int32_t n_bounces);

/* Rays per bounce of the bounce-by-bounce steps taken while profiling was on
 * (DR_OPT_PROFILE; single-scene contexts, outside frame capture): HOST
 * output rays[2 * n_bounces], row 0 the closest-hit rays of bounce k, row 1
 * the shadow (next-event) rays made at bounce k, column k - 1 = bounce k,
 * accumulated since the last dr_get_profile (which clears them).  Counting
 * waits for each profiled step to finish.  No synchronisation here.
 * Errors: INVALID_ARG (n_bounces outside 1..16). */
int dr_get_bounce_rays(dr_ctx* ctx, uint64_t* rays, int32_t n_bounces);

/* One frame of the per-frame loop: n_steps Evolve steps (Alg. 2, as
 * dr_step) followed by the splat of their records (as dr_splat), issued as
 * one CUDA graph that is captured on the first call and replayed by later
 * calls with the same configuration (recaptured automatically when the
 * chains, scene, parameters or options change).  The step index is kept in
 * device memory so every replay draws new Philox numbers.  Requires that
 * the context was created on a created (non-default) stream.  Asynchronous.
 * Errors: STATE (no chains; default stream), CUDA, OOM. */
int dr_frame(dr_ctx* ctx, uint32_t n_steps);

/* BVH construction used by later dr_scene_upload calls:
 * DR_BVH_PLOC (default; parallel locally-ordered clustering of the
 * Morton-ordered triangles with search radius `radius`, 1..256, default 16)
 * or DR_BVH_LBVH (linear BVH, Karras 2012; radius ignored).  Both produce
 * the same node layout.  A clustered tree taller than the traversal stack
 * allows (exact ties among many triangle boxes, e.g. coincident triangles,
 * make the clustering merge one pair per pass) is replaced by the linear
 * BVH of the same scene.  Errors: INVALID_ARG. */
enum { DR_BVH_LBVH = 0, DR_BVH_PLOC = 1 };
int dr_set_bvh_builder(dr_ctx* ctx, int32_t builder, int32_t radius);

/* Splat without allocating: the paper has no counterpart to this entry point;
 * it exists for callers that cannot call cudaMalloc (for example a render
 * loop held to a fixed device-memory budget, code running where another
 * framework owns the device's allocator, or code that must not pay for the
 * device-wide synchronisation cudaMalloc / cudaFree can cause).
 * It computes what dr_splat_records computes: accum[pix * 3 + c] += the FP64
 * sum of the records' values, sorted by pixel (stable, so the sum order is
 * the records' order), without a context.
 *   recs    DEVICE, M records of 16 bytes (uint32 pixel, float r, g, b);
 *           only read.
 *   M       0 .. DR_NOALLOC_MAX_RECORDS; larger M is rejected with
 *           DR_ERR_INVALID_ARG (split the records into batches).
 *   n_pix   number of pixels, 1 .. 2^31 - 2; pixel indices should be
 *           < n_pix.  A record at or above it is skipped (every other
 *           pixel's sum stays exact) and marks the call as failed, which
 *           dr_splat_records_noalloc_status reports.
 *   accum   DEVICE FP64 [n_pix * 3], added to (not cleared).
 *   cuda_stream  stream to issue on (NULL: legacy default stream).
 * All pointers must belong to the current CUDA device.  The scratch is a
 * fixed array of about 2.1 MB in this library's device memory, present on
 * every GPU that loads the library until the process exits; it calls no
 * cudaMalloc, cudaFree or allocating routine.  A call outside stream
 * capture looks up the array's device address (so after a device reset the
 * next such call finds it again); a call during capture uses the address
 * the last call outside capture found, so make the first call on a device
 * before any stream capture.  Every call on a device shares the one array,
 * so calls that overlap on the GPU (for example on two streams at once)
 * race; issue them in order on one stream, or synchronise between them.
 * Asynchronous.  Errors: INVALID_ARG, CUDA. */
enum { DR_NOALLOC_MAX_RECORDS = 65536 };
int dr_splat_records_noalloc(const void* recs, int64_t M, int32_t n_pix, double* accum, void* cuda_stream);

/* Outcome of the last dr_splat_records_noalloc call on the current device
 * (its scratch array holds one error word, cleared by every call): waits
 * for cuda_stream, then returns DR_OK, or DR_ERR_DEVICE_CHECK if a record's
 * pixel index was >= n_pix.  Not during stream capture (STATE).
 * Errors: STATE, CUDA, DEVICE_CHECK. */
int dr_splat_records_noalloc_status(void* cuda_stream);

/* Resolve (Alg. 3) on caller buffers, without a context: out[i] =
 * k0 / tour_count * accum[i] for i < n, in FP64, rounded to FP32.  For
 * replicas that summed their FP64 accumulators and tour counts (one run
 * over the union of their chains).  accum DEVICE FP64 [n], out DEVICE FP32
 * [n], cuda_stream may be NULL.  When tour_count = 0 it writes zeros and
 * returns DR_ERR_STATE (as dr_resolve).  Asynchronous otherwise.
 * Errors: INVALID_ARG (NULL pointer, n < 0, k0 not finite), STATE, CUDA. */
int dr_resolve_accum(const double* accum, int64_t n, uint64_t tour_count, double k0, float* out, void* cuda_stream);

/* The initial samples' sum of p (FP64, summed in a fixed block order) and
 * their count, from the last dr_chains_init that estimated p_lambda
 * (p_lambda = p_sum / n).  Replicas add these over ranks and pass the totals
 * to dr_k0_from_p_sum, so every rank uses the k0 of the pooled samples.
 * HOST outputs.  Errors: INVALID_ARG, STATE (no estimate: k0 was given, or
 * the chains came from a checkpoint). */
int dr_get_p_sum(dr_ctx* ctx, double* p_sum, uint64_t* n);

/* k0 = p_lambda / (m dt) with p_lambda = p_sum / n (Eq.
 * killing-rate-constant; m and dt from prm, a HOST pointer).  Host
 * arithmetic only.  Errors: INVALID_ARG (n = 0, p_sum not positive and
 * finite, m dt not positive, NULL pointer). */
int dr_k0_from_p_sum(double p_sum, uint64_t n, const dr_params* prm, double* k0);

/* Shape of the current chain state (HOST outputs, any may be NULL): number
 * of chains N, PSS dimension d and max path length L; the sizes callers of
 * dr_readback_state must allocate for (e.g. after dr_state_load).
 * Errors: STATE when no chains exist. */
int dr_get_chain_shape(dr_ctx* ctx, uint64_t* n_chains, int32_t* dim, int32_t* max_path_len);

#ifdef __cplusplus
}
#endif

#endif /* DIFFRESTORE_H_ */
