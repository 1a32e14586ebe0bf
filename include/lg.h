/*
 * lg.h -- C-ABI of liblgdock: batched flexible-ligand docking and scoring on
 * one GB300 (sm_103a).
 *
 * The library implements the dock-and-score step of the EXSCALATE platform
 * (paper Sec. 3.1): every ligand is docked into a rigid binding site by a
 * greedy optimisation with multiple restarts, driven by a geometric (steric)
 * score, with the ligand made flexible through its torsional bonds, which are
 * processed one after the other; the ligand's score is that of its best pose.
 * The binding site is constant for the life of the application and is loaded
 * once (Sec. 3.2), and a ligand's own description is all that docking it needs
 * (Sec. 3.2), so the calls below take a pocket handle plus a batch of ligand
 * descriptions.  Results depend only on (ligand uid, seed, pocket, parameters),
 * so a pose can be regenerated on demand from the stored score (Sec. 4.1).
 *
 * Concrete readings of the method (restart pose from Philox4x32-10 and
 * Shoemake rotations, 36 torsion steps of 10 degrees, intra-ligand clash
 * distance, trilinear grid scoring, tie-breaks) are stated at lg_dock_batch.
 *
 * Conventions for every call:
 *   - Return value: LG_OK or one of the LG_E* codes; lg_last_error() gives a
 *     message (per calling thread).  No C++ exception crosses this boundary.
 *   - Pointers are host or device pointers as the struct's `mem` field says.
 *     Device pointers must be CUDA device (or managed) memory of the device the
 *     context was created on.  Arrays are dense, with the element types given.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Nothing the caller passes is retained after a call returns, except where
 *     stated (asynchronous device-memory docking, stream submission).
 */
#ifndef LG_H
#define LG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define LG_OK 0
#define LG_EINVAL 1     /* bad argument or malformed ligand */
#define LG_ENOMEM 2     /* device or host allocation failed */
#define LG_EAGAIN 3     /* queue full / not enough free device memory yet */
#define LG_ETIMEOUT 4   /* a bounded wait ran out */
#define LG_ECUDA 5      /* a CUDA runtime call failed */
#define LG_ENOPOCKET 6  /* unknown pocket id */

#define LG_MEM_HOST 0
#define LG_MEM_DEVICE 1

#define LG_MODE_BATCHED 0 /* persistent, cost-sorted, one launch per batch */
#define LG_MODE_PLAIN 1   /* one launch per ligand, one warp per restart */

#define LG_MAX_ATOMS 128  /* atoms per ligand */
#define LG_MAX_ROT 32     /* torsional bonds per ligand */
#define LG_MAX_PASSES 8
#define LG_MAX_RESTARTS 1024
#define LG_ANGLE_STEPS 36 /* torsion steps per bond (10 degrees each) */
#define LG_NUM_TYPES 5    /* atom types C, N, O, S, Cl */

typedef struct lg_ctx lg_ctx;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  The context owns every device
 * allocation the library makes (pockets, staging and scratch buffers) and the
 * serving worker.  Errors: LG_EINVAL (bad device), LG_ECUDA. */
int lg_create(int device, lg_ctx **out);

/* Destroy a context: stops the serving worker (pending requests fail), frees
 * every pocket and buffer.  Safe on NULL. */
void lg_destroy(lg_ctx *ctx);

/* Message of the last error returned to the calling thread (never NULL). */
const char *lg_last_error(lg_ctx *ctx);

/* ---------------------------------------------------------------- pockets */

/* A rigid binding site (Sec. 3.2: fetched once, stored where each
 * implementation sees fit -- here packed per grid cell in device memory).
 * Grids are n^3 FP32 values, x fastest: node (i,j,k) is at origin + h*(i,j,k)
 * and its value at phi[(k*n + j)*n + i].
 *   phi_o          pocket-overlap field that drives the torsion sweep
 *   phi_v, phi_e   vdW-like potential and electrostatic potential per unit
 *                  charge, used by the final pose score
 *   pocket_points  n_pp node indices (i,j,k) where restart poses are centred
 *   type_w         per-type multipliers of phi_v (C, N, O, S, Cl)
 *   k_out          slope of the penalty for atoms outside the grid box */
typedef struct {
    int32_t n;
    float h;
    float origin[3];
    const float *phi_o;
    const float *phi_v;
    const float *phi_e;
    int32_t n_pp;
    const int32_t *pocket_points;
    float type_w[LG_NUM_TYPES];
    float k_out;
} lg_pocket_desc;

/* Copy a pocket (host pointers) into device memory owned by the context and
 * return its id.  The caller's buffers may be freed on return.  Requires
 * 2 <= n <= 512, h > 0, n_pp >= 1 and every pocket point inside the grid.
 * The three grids go to the device as they are (12 bytes per node) and a
 * kernel packs them into per-node cells of trilinear coefficients (32 bytes
 * per node for phi_o, 64 for phi_v and phi_e side by side; FP64 differences
 * of the grid values rounded to FP32, see lg_diag_pocket_cells); option
 * "pocket_pack_host" = 1 packs them on the host instead, with the same
 * arithmetic and the same result, and uploads the cells.
 * L2 residency (the paper keeps the site in texture memory, Sec. 3.2): the
 * call sizes the context's persisting L2 set-aside for the largest loaded
 * pocket's overlap cells (32 bytes per node; within the device's limit; a
 * context setting that ends with the context), and every later docking
 * launch against one pocket carries an access-policy window that marks that
 * pocket's cells persisting (option "l2_window").  The window never changes a
 * result.  Errors: LG_EINVAL, LG_ENOMEM, LG_ECUDA. */
int lg_pocket_load(lg_ctx *ctx, const lg_pocket_desc *d, int32_t *pocket_id);

/* Free a pocket.  The caller must not have docking in flight on it.
 * Errors: LG_ENOPOCKET. */
int lg_pocket_unload(lg_ctx *ctx, int32_t pocket_id);

/* ---------------------------------------------------------------- ligands */

/* A batch of L ligands in CSR structure-of-arrays layout (Sec. 4.1: each
 * ligand is described by atom positions, types and bonds).
 *   atom_off[L+1]   atoms of ligand l are atom_off[l] .. atom_off[l+1]-1
 *   x,y,z,q [A]     FP32 coordinates (A) and partial charges
 *   type [A]        0..4 = C, N, O, S, Cl
 *   parent [A]      local index of the atom's parent in the ligand's bond tree,
 *                   -1 for local atom 0; atoms must be in depth-first preorder
 *                   (parent[i] < i and every subtree a contiguous index range)
 *   rot_off[L+1]    torsional bonds of ligand l are rot_off[l] .. rot_off[l+1]-1
 *   rot_child [R]   a torsional bond is named by its child atom b (local index):
 *                   the bond (parent[b], b); strictly ascending per ligand
 *   uid [L]         ligand identity; the random restart poses depend on it only
 * A ligand that breaks these rules gets status LG_EINVAL and the others run.
 * Limits: 1 <= atoms <= LG_MAX_ATOMS, torsional bonds <= LG_MAX_ROT. */
typedef struct {
    int32_t L;
    int32_t mem; /* LG_MEM_HOST or LG_MEM_DEVICE, for every pointer below */
    const int32_t *atom_off;
    const float *x, *y, *z, *q;
    const uint8_t *type;
    const int16_t *parent;
    const int32_t *rot_off;
    const int16_t *rot_child;
    const uint64_t *uid;
} lg_ligand_batch;

/* Docking parameters (Sec. 3.1: restarts of the greedy optimisation; the
 * paper's run used 256 initial poses per ligand).
 *   restarts     1..LG_MAX_RESTARTS random initial poses per ligand
 *   passes       0..LG_MAX_PASSES sweeps over all torsional bonds
 *   angle_steps  must be LG_ANGLE_STEPS (36 steps of 10 degrees)
 *   seed         64-bit key of the restart-pose random stream
 *   d_clash      minimum distance (A) between a moving atom and a fixed atom
 *                three or more bonds away; > 0
 *   mode         LG_MODE_BATCHED or LG_MODE_PLAIN
 *   plain_streams  streams the plain mode spreads its launches over (1..64;
 *                0 = 8); ignored in batched mode
 *   max_atoms, max_rot  optional declared maxima over the batch (0 = the
 *                library limits).  They size the kernels' shared memory: a
 *                smaller declaration lets more CTAs share an SM.  Ligands
 *                above a declared maximum get status LG_EINVAL.  For host
 *                batches the library also measures the maxima itself.
 *   cluster_rmsd, rescore_top  pose ranking (paper Sec. 3.1, steps 3-4), off
 *                when cluster_rmsd = 0 and rescore_top is 0 or >= restarts:
 *                the restart poses are ordered by geometric score (the total
 *                overlap of the pose, higher first, lower restart on ties) and
 *                clustered greedily -- a pose within cluster_rmsd A RMSD (no
 *                superposition) of an earlier cluster leader joins the first
 *                such leader, else it leads a new cluster; the ranking lists
 *                the leaders, then the other poses, in that order; the first
 *                rescore_top ranked poses (all when 0) are rescored and the
 *                lowest score among them is the ligand's result.  The paper's
 *                setting is 256 restarts, 3 A and the top 30.  Ranking keeps
 *                every restart's final pose in device scratch (12 bytes per
 *                atom and restart for each ligand docked at once) and needs
 *                shared memory growing as restarts^2 / 16 bytes (68 KB at
 *                1,024 restarts), which can lower the kernels' occupancy.
 *   rigid_steps, rigid_shift  rigid greedy refinement (the paper's greedy
 *                optimisation read broadly, Sec. 3.1), off when rigid_steps =
 *                0: after each torsion pass, rigid_steps (0..LG_MAX_RIGID_STEPS)
 *                moves of the whole ligand, each the best of 13 candidates by
 *                the total overlap of all atoms (lowest candidate on ties):
 *                0 stay; 1..6 shift by +rigid_shift, -rigid_shift (A, >= 0)
 *                along x, y, z; 7..12 turn by +10, -10 degrees about the x, y, z
 *                axes through the ligand's centroid.  Candidate sums are FP64
 *                over FP32 lookups. */
#define LG_MAX_RIGID_STEPS 16
typedef struct {
    int32_t restarts;
    int32_t passes;
    int32_t angle_steps;
    uint64_t seed;
    float d_clash;
    int32_t mode;
    int32_t plain_streams;
    int32_t max_atoms;
    int32_t max_rot;
    float cluster_rmsd;
    int32_t rescore_top;
    int32_t rigid_steps;
    float rigid_shift;
} lg_dock_params;

/* Caller-owned outputs (all with the location given by `mem`).
 *   score [L]          FP64 score E of the best pose (lower is better), NaN on error
 *   best_restart [L]   restart index of the best pose, -1 on error
 *   tors_idx           optional: torsion step (0..35) chosen at each decision of
 *                      the best restart, passes*rot_off[l] + pass*R_l + k
 *   pose               optional: best pose, 3*atom_off[l] + 3*i + {x,y,z} (A)
 *   status [L]         LG_OK or LG_EINVAL per ligand
 *   restart_score      optional: E of every restart, l*restarts + r
 *   restart_tors       optional: steps of every restart,
 *                      restarts*passes*rot_off[l] + (r*passes + pass)*R_l + k
 *   rank, leader, restart_geo  optional, with pose ranking on: the ranked
 *                      restarts (l*restarts + position), each restart's cluster
 *                      leader and geometric score (l*restarts + r)
 *   restart_rigid      optional, with rigid refinement on: the candidate taken
 *                      at every rigid move of every restart,
 *                      ((l*restarts + r)*passes + pass)*rigid_steps + j
 *   decision_rank      optional (not with the serving loop nor lg_dock_multi's
 *                      ligand-major order: LG_EINVAL): for every torsion
 *                      decision of every restart (the layout of restart_tors),
 *                      1 + the number of steps ranked before the chosen one by
 *                      overlap score (higher score, or equal score and lower
 *                      step): the steps whose clash check a method cannot skip.
 *                      Decisions skipped after convergence repeat the bond's
 *                      previous decision and its rank, with bit 7 (0x80) set
 *                      to mark them skipped (the rank is the low 7 bits); a
 *                      bond that moves no atom ranks 1.  For accounting (work
 *                      per decision, and the work the exact stops skip). */
typedef struct {
    int32_t mem;
    double *score;
    int32_t *best_restart;
    uint8_t *tors_idx;
    float *pose;
    int32_t *status;
    double *restart_score;
    uint8_t *restart_tors;
    int32_t *rank;
    int32_t *leader;
    double *restart_geo;
    uint8_t *restart_rigid;
    uint8_t *decision_rank;
} lg_dock_result;

/* Dock and score a batch of ligands against one pocket (paper Sec. 3.1).
 *
 * Per (ligand, restart r):
 *   1. pose: Philox4x32-10 (key = seed, counter = (uid_lo, uid_hi, r, 0)) gives
 *      x0..x3; u_i = (x_i >> 8) * 2^-24; Shoemake's uniform quaternion from
 *      (u0, u1, u2) gives R; the pocket point is number ((x3 >> 8) * n_pp) >> 24;
 *      atoms are placed at R (x - centroid) + pocket point.
 *   2. sweep: `passes` times, each torsional bond in ascending child order:
 *      the atoms hanging below the child turn about the bond axis through the
 *      child by each of 36 steps of 10 degrees; a step's overlap score is the
 *      sum of phi_o (trilinear) over those atoms; a step is admissible when it
 *      is step 0 or no moved atom comes closer than d_clash to an atom outside
 *      the child's subtree that is three or more bonds away; the admissible
 *      step with the highest overlap (lowest step on ties) is applied.
 *   3. score: E = sum over atoms of type_w*phi_v + q*phi_e at the position
 *      clamped to the grid box, plus k_out times the distance outside the box;
 *      per-atom terms in FP32, sum in FP64.
 *   4. best: the lowest E wins, the lowest restart on ties.  With pose
 *      ranking on (cluster_rmsd > 0, or 0 < rescore_top < restarts) the best
 *      is instead the lowest E among the first rescore_top ranked poses; see
 *      lg_dock_params and lg_dock_result for the ranking's definition.
 * Geometry and lookups run in FP32.
 *
 * Memory: if the batch and result are device memory the call is asynchronous
 * on `stream` and the caller keeps every buffer alive until the stream
 * reaches the end of the call; otherwise the library stages through its own
 * device buffers and returns after the results are in host memory.  Calls on
 * one context share its scratch buffers: the library makes each call's stream
 * wait for the previous call's device work, so asynchronous calls on
 * different streams run one after the other on the device.
 * Errors: LG_EINVAL (bad parameters or sizes; per-ligand problems go to
 * status[] instead), LG_ENOPOCKET, LG_ENOMEM, LG_ECUDA. */
int lg_dock_batch(lg_ctx *ctx, int32_t pocket_id, const lg_ligand_batch *batch, const lg_dock_params *params,
                  lg_dock_result *out, void *stream);

/* Dock one batch against several loaded pockets: the screening campaign's
 * pattern, a ligand library against every binding site (paper Sec. 1 and 4:
 * 15 binding sites).  Results are those of n_pockets lg_dock_batch calls, bit
 * for bit: outs[k] receives the results for pocket_ids[k].  The per-ligand
 * preparation (validation, subtree ends, centroid, cost order) runs once for
 * all pockets.  Visiting order (context option "multi_order"): pocket-major,
 * the default, docks the batch against each pocket in turn with one
 * persistent launch per pocket, so only one pocket's grids need to be in L2;
 * ligand-major is one launch in which a CTA docks its ligand against every
 * pocket.
 *   - Batched mode only (params->mode = LG_MODE_BATCHED).
 *   - Every outs[k] has the same mem and the same set of optional outputs.
 *   - Memory and errors as lg_dock_batch.  1 <= n_pockets <= 64. */
#define LG_MAX_MULTI_POCKETS 64
int lg_dock_multi(lg_ctx *ctx, const int32_t *pocket_ids, int32_t n_pockets, const lg_ligand_batch *batch,
                  const lg_dock_params *params, lg_dock_result *outs, void *stream);

/* Ligand flattening (paper Sec. 3.1, step 1: before docking, the torsional
 * bonds are turned to maximise the sum of the distances between all atom
 * pairs; protein independent, so done once per ligand for every pocket).
 * Reading: the docking's greedy sweep without a pocket -- for pass =
 * 0..passes-1 and each torsional bond in ascending child order, the 36 steps
 * of 10 degrees turn the bond's moving atoms; the admissible step (the clash
 * rule of lg_dock_batch with d_clash) with the largest sum of pairwise
 * distances is applied, the lowest step on ties.  The ligand stays in its
 * input frame.  Distances are FP32, summed in FP32 within 32 pairs and in FP64
 * across them.
 *   passes       0..LG_MAX_PASSES sweeps over the torsional bonds
 *   angle_steps  must be LG_ANGLE_STEPS
 *   d_clash      clash distance (A), > 0
 *   max_atoms, max_rot  optional declared maxima (0 = the library limits) */
typedef struct {
    int32_t passes;
    int32_t angle_steps;
    float d_clash;
    int32_t max_atoms;
    int32_t max_rot;
} lg_flatten_params;

/* Caller-owned outputs (location given by `mem`):
 *   xyz [3*A]      flattened coordinates, 3*atom_off[l] + 3*i + {x,y,z}; a
 *                  rejected ligand's input coordinates
 *   tors           optional: step applied at each decision,
 *                  passes*rot_off[l] + pass*R_l + k
 *   dsum [L]       optional: FP64 sum of all pairwise distances of the result
 *                  (NaN for a rejected ligand)
 *   status [L]     LG_OK or LG_EINVAL per ligand (the checks of lg_dock_batch) */
typedef struct {
    int32_t mem;
    float *xyz;
    uint8_t *tors;
    double *dsum;
    int32_t *status;
} lg_flatten_result;

/* Flatten a batch.  Memory rules as lg_dock_batch (asynchronous on `stream`
 * when batch and result are device memory).  Errors: LG_EINVAL, LG_ENOMEM,
 * LG_ECUDA. */
int lg_flatten_batch(lg_ctx *ctx, const lg_ligand_batch *batch, const lg_flatten_params *params,
                     lg_flatten_result *out, void *stream);

/* Allocation-free docking (the paper has no counterpart to this call).
 * Some callers cannot let a library allocate device memory: applications that
 * give all device memory to their own pool allocator at start-up (a cudaMalloc
 * from outside the pool fails or fragments it), and latency-critical callers
 * that cannot accept the device-wide synchronisation cudaMalloc / cudaFree may
 * cause.  This call docks exactly like lg_dock_batch in LG_MODE_BATCHED but
 * allocates nothing: the scratch of the batched kernels lives in a fixed
 * device array of LG_NOALLOC_SCRATCH_BYTES that every device loading the
 * library holds until the process exits.
 *   - batch and out must be device memory (host staging would allocate); the
 *     call is asynchronous on `stream` like lg_dock_batch.
 *   - The scratch needs about 32 + 2 * max_rot bytes per ligand (max_rot = 32
 *     when 0) plus 1 KiB; larger batches are rejected with LG_EINVAL.
 *   - Every call looks up the array's device address with the context's
 *     device current (a host-side lookup).  The first call on a device may
 *     also load the library's device code there: make that first call before
 *     any stream capture.
 *   - Every call shares the array and finds the previous call's contents in
 *     it; the call clears the counters that must start at zero.  Calls whose
 *     work overlaps on the GPU race on the array: order them on one stream.
 *   - The pocket must already be loaded (lg_pocket_load allocates).
 *   - Pose ranking (cluster_rmsd > 0, or 0 < rescore_top < restarts) needs
 *     per-CTA pose slots that the fixed array does not hold: LG_EINVAL.
 * Errors: LG_EINVAL, LG_ENOPOCKET, LG_ECUDA. */
#define LG_NOALLOC_SCRATCH_BYTES (4u << 20)
int lg_dock_batch_noalloc(lg_ctx *ctx, int32_t pocket_id, const lg_ligand_batch *batch, const lg_dock_params *params,
                          lg_dock_result *out, void *stream);

/* Given poses to score (step 3 above alone).
 *   atom_off[L+1], xyz[3*A] (A, interleaved), q[A], type[A]. */
typedef struct {
    int32_t L;
    int32_t mem;
    const int32_t *atom_off;
    const float *xyz;
    const float *q;
    const uint8_t *type;
} lg_pose_batch;

/* Score L given poses against a pocket: energies[L] (FP64, same `mem` as the
 * batch).  Synchronous for host memory, stream-ordered for device memory.
 * Errors: LG_EINVAL, LG_ENOPOCKET, LG_ENOMEM, LG_ECUDA. */
int lg_score_poses(lg_ctx *ctx, int32_t pocket_id, const lg_pose_batch *batch, double *energies, void *stream);

/* ---------------------------------------------------------------- serving */

#define LG_REQ_QUEUED 0
#define LG_REQ_RUNNING 1
#define LG_REQ_DONE 2
#define LG_REQ_FAILED 3

/* Submit a docking request to the context's serving loop (the paper streams
 * a chemical library through a fixed binding site, Sec. 3.2-3.3).  The batch
 * must be host memory; it is copied before the call returns, so the caller
 * may free it.  `out` must be host memory and stay alive until the request is
 * DONE or FAILED.  Requests are admitted to the device when enough free
 * device memory and in-flight slots exist, and their ligands share the device
 * with the other requests in flight.  Never blocks on the GPU.
 *
 * By default (option "serve_device_loop" = 1) the requests are served by a
 * device-resident loop: one persistent launch takes ligands, one per CTA, in
 * admission order from a ring of request descriptors that the host fills with
 * copies, docks each against its request's own pocket and writes the results
 * straight into the request's pinned output image, and the CTA that finishes
 * a request's last ligand raises the request's completion flag in mapped host
 * memory.  A request that arrives while others run is docked as soon as CTAs
 * free up.  The loop serves one kind of request at a time (restarts, passes,
 * seed, clash distance, ranking and rigid settings, optional outputs, atom
 * and torsion maxima up to 64/128 and 16/32): a request of another kind waits
 * until the requests in flight finish, and the loop is then set up for it.
 * Its CTAs leave after "serve_loop_idle_ms" without a ligand to claim, so an
 * idle loop ends by itself; lg_stats.serve_loop_status says how the last
 * launch ended.  With "serve_device_loop" = 0 a host worker instead merges
 * queued requests into ordinary batched launches on up to
 * "serve_max_inflight" streams.
 * Errors: LG_EINVAL, LG_ENOPOCKET, LG_EAGAIN (host queue full), LG_ENOMEM. */
int lg_stream_submit(lg_ctx *ctx, int32_t pocket_id, const lg_ligand_batch *batch, const lg_dock_params *params,
                     lg_dock_result *out, uint64_t *ticket);

/* State of a request (LG_REQ_*) and, once DONE, its submit-to-done latency in
 * seconds.  Never blocks.  Errors: LG_EINVAL (unknown ticket). */
int lg_stream_poll(lg_ctx *ctx, uint64_t ticket, int32_t *state, double *latency_s);

/* Block until the request is DONE or FAILED, at most timeout_ms milliseconds.
 * Errors: LG_ETIMEOUT, LG_EINVAL (unknown ticket), LG_ECUDA (request FAILED). */
int lg_stream_wait(lg_ctx *ctx, uint64_t ticket, int32_t timeout_ms);

/* ---------------------------------------------------------------- introspection */

/* Figures of the lg_dock_batch calls on this context.  With timing on
 * (lg_set_option "timing" = 1, which also clears the totals) every call
 * brackets its docking kernel(s) with CUDA events on the call's stream;
 * lg_get_stats waits for those events and reports the last call's device time
 * and the sum over the calls since timing was switched on. */
typedef struct {
    float dock_ms;        /* device time of the last call's docking kernel(s) */
    int32_t dock_calls;   /* timed calls since timing was switched on */
    double dock_ms_total; /* their summed device time */
    int32_t launches;     /* kernels launched by the last call */
    int32_t grid;         /* CTAs of the docking kernel (batched mode) */
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
    int32_t smem_bytes;   /* dynamic shared memory per CTA */
    int32_t graph;        /* last call: 2 captured a CUDA graph, 1 replayed one, 0 launched directly */
    int32_t serve_loop_status;   /* device-resident serving loop: how its last launch ended (LG_OK after a
                                    stop, LG_ETIMEOUT after its idle limit, LG_EINVAL for a bad work item;
                                    -1 while running or never launched) */
    int32_t restart_lanes;       /* lanes per restart of the last call's first batched launch (32: plain mode) */
    int64_t l2_window_bytes;     /* L2 access-policy window of the last docking launch (0: none) */
    int64_t l2_persist_bytes;    /* persisting L2 set-aside of the context (0: none) */
    int64_t serve_loop_launches; /* launches of the device-resident serving loop */
    int64_t serve_loop_items;    /* ligands it has docked */
    int64_t serve_loop_switches; /* its switches between restart tiles (option "serve_loop_lanes" = 0) */
} lg_stats;

int lg_get_stats(lg_ctx *ctx, lg_stats *out);

/* Context options: "timing" (0/1, default 0), "warps_per_cta" (0 = the
 * autotuner's or the default choice, else 1..4 for every batched launch; up
 * to 8 or 16 with 8 or 16 lanes per restart), "restart_lanes" (0 = the
 * autotuner's or the default choice, else 2, 4, 8 or 16 lanes per restart --
 * 16, 8, 4 or 2 restart slots per warp -- for every single-pocket batched
 * launch without pose ranking or decision ranks; the others always use 4),
 * "autotune" (0/1, default 1; setting it clears the tuned choices: with it on,
 * the first batched call of a (size class, restarts, passes, atom and torsion
 * maxima, features) combination times the candidate tiles -- (lanes per
 * restart, warps per CTA) = (4, 4), (4, 2), (4, 1), (2, 2), (2, 1), (8, 4),
 * (8, 2), or (4, 4), (4, 2), (4, 1) where only 4 lanes per restart exist --
 * on the same even sample of that class's ligands (16 waves of the widest
 * grid, at least 4,096) and keeps the fastest; a batch that fits in one wave
 * instead takes 16 (else 8, else 4) lanes per restart with every restart of a
 * ligand in flight at once, untuned; results never depend on the choice), "graphs" (0/1/2, default 2: an lg_dock_batch call with device
 * batch and result on a non-default stream is captured, preparation and
 * docking kernels together, as a CUDA graph -- with 2 when its arguments
 * recur, i.e. from the second call with the same arguments on, with 1 on the
 * first call -- and replayed when a later call has the same arguments; 0: no
 * graphs; with timing on, a graph call's device time spans the preparation
 * kernels too; setting the option drops the captured graphs), "size_classes" (0/1, default 1: a batch whose atom maximum exceeds
 * 64 is docked by one launch per size class -- atoms <= 32, <= 64, more --
 * each with shared memory for its own maximum), "serve_max_inflight" (requests on the device at once, default 8),
 * "serve_mem_reserve_mb" (free device memory the server leaves untouched,
 * default 1024), "serve_max_merge" (ligands per merged batch, default 4,096),
 * "serve_cross_pocket" (0/1, default 0: merge requests aimed at different
 * pockets into one launch, each ligand docked against its own request's
 * pocket), "multi_order" (lg_dock_multi's visiting order: 0 =
 * pocket-major, the default; 1 = ligand-major, a CTA docks one ligand against
 * every pocket in turn), "l2_window" (0/1, default 1: every docking launch
 * against one pocket marks that pocket's overlap cells persisting in the L2
 * set-aside that lg_pocket_load reserves), "serve_device_loop" (0/1, default
 * 1: the device-resident loop serves the requests, see lg_stream_submit;
 * changing it stops the serving worker -- requests on the device finish,
 * queued ones fail -- and the next submission starts one of the other kind),
 * "serve_loop_idle_ms" (1..60000, default
 * 100: how long a CTA of the loop waits for a ligand before it leaves; the
 * first CTA to leave ends the launch as a whole), "serve_loop_lanes" (0, 4
 * or 16, default 0: lanes per restart of the loop's restart tile; at 16 a
 * CTA holds every restart of its ligand at once, one CTA per SM, which about
 * halves each ligand's time in the loop at light load but lowers the loop's
 * peak rate; 4 is the throughput tile; 0 switches between them by the
 * backlog -- 16 while the ligands of the requests on the device stay within
 * eight waves of the 16-lane loop, 4 above that until the backlog has stayed
 * within one wave for 5 ms; a switch stops the running launch, whose
 * CTAs leave after their current ligand, and relaunches with the other tile;
 * requests that rank poses always use 4; changing the option stops the
 * serving worker as "serve_device_loop" does).
 * Errors: LG_EINVAL. */
int lg_set_option(lg_ctx *ctx, const char *key, int64_t value);

/* The autotuner's cached choices as JSON text, to carry them to another
 * context or process on the same kind of GPU:
 *   {"device": "<name>", "sms": <SM count>, "entries": [[size class,
 *    restarts, passes, atom maximum, torsion maximum, ranking + 2 * decision
 *    ranks, rigid, kind, lanes per restart, warps per CTA], ...]}
 * (an entry of 9 integers, without the lanes per restart, means 4)
 * lg_tune_export writes the text, NUL-terminated, into buf (cap bytes,
 * caller-owned) and sets *len to its length without the NUL; when cap is too
 * small it writes nothing, sets *len and returns LG_EINVAL (buf may be NULL
 * with cap 0 to ask for the length).  lg_tune_import adds the entries of such
 * a text to the context's cache; a text from another device name or SM
 * count, or one that does not parse, is refused with LG_EINVAL and the cache
 * is left unchanged.  Setting the "autotune" option clears the cache. */
int lg_tune_export(lg_ctx *ctx, char *buf, int64_t cap, int64_t *len);
int lg_tune_import(lg_ctx *ctx, const char *text);

/* ---------------------------------------------------------------- diagnostics */

/* Philox4x32-10 of n (counter, key) pairs on the device (device pointers:
 * ctr[4n], key[2n], out[4n] as uint32).  use_curand = 0 runs the library's own
 * generator, 1 runs cuRAND's curand_Philox4x32_10 for comparison.
 * Synchronous.  Errors: LG_EINVAL, LG_ECUDA. */
int lg_diag_philox(lg_ctx *ctx, int32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                   int32_t use_curand);

/* Measured FP32 FMA throughput of the context's device in TFLOP/s (the
 * roofline's denominator for the FP32-bound docking kernels): reps timed
 * launches (1..100, after one warm-up) of a kernel whose threads run 8
 * independent FMA chains, 8 CTAs of 256 threads per SM, 2 FLOP per FMA;
 * *tflops gets the best launch, *seconds (may be NULL) the timed total.
 * Synchronous.  Errors: LG_EINVAL, LG_ECUDA. */
int lg_diag_fp32_peak(lg_ctx *ctx, int32_t reps, double *tflops, double *seconds);

/* The packed cells of a loaded pocket copied to host memory (caller-owned):
 * cell_o[8 n^3] (overlap grid) and cell_ve[16 n^3] (vdW then electrostatic
 * coefficients per node), node (i, j, k) at (k n + j) n + i, coefficients
 * (c000, c100, c010, c001, c110, c101, c011, c111) of the cell's trilinear
 * polynomial in the cell's local coordinates (see lg_pocket_load).
 * Synchronous.  Errors: LG_EINVAL (unknown pocket), LG_ECUDA. */
int lg_diag_pocket_cells(lg_ctx *ctx, int32_t pid, float *cell_o, float *cell_ve);

#ifdef __cplusplus
}
#endif
#endif /* LG_H */
