// Internal declarations shared by the runtime (lg_runtime.cu, lg_serve.cu) and
// the kernels (lg_kernels.cu).  Not part of the public ABI (include/lg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lg.h"

namespace lg {

// Device view of a loaded pocket.
//
// Frames.  Kernels keep positions in "centred grid units": x_g = (x_world -
// center) / h, with center the middle of the grid box, so |x_g| <= (n-1)/2 for
// atoms inside the box.  The grid index of a position is x_g + c0, c0 = (n-1)/2:
// node (i,j,k) sits at index (i,j,k).  Rotations commute with the uniform
// scaling, distances are compared in grid units (d_clash^2 / h^2).
//
// Cells.  For every node (i,j,k), i,j,k in [0, n-1], the 8 coefficients of the
// trilinear polynomial through the values at (i+a, j+b, k+c), a,b,c in {0,1}
// (indices clamped to n-1, so the last layer repeats the edge):
//   p(fx,fy,fz) = c0 + c1 fx + c2 fy + c3 fz + c4 fx fy + c5 fx fz + c6 fy fz + c7 fx fy fz
// stored as two float4 (c0..c3, c4..c7): one 32-byte sector per lookup.
// cell_ve holds 16 coefficients per node: phi_v's then phi_e's.
struct PocketDev {
    int n;
    float h, inv_h, c0, gmax;  // gmax = n - 1
    float3 center;             // world position of the box centre
    const float4 *cell_o;      // 2 float4 per node
    const float4 *cell_ve;     // 4 float4 per node
    const float4 *pp;          // pocket points in centred grid units (x, y, z, 0)
    int n_pp;
    float type_w[LG_NUM_TYPES];
    float k_out;
};

struct BatchDev {
    int L;
    const int32_t *atom_off;
    const float *x, *y, *z, *q;
    const uint8_t *type;
    const int16_t *parent;
    const int32_t *rot_off;
    const int16_t *rot_child;
    const uint64_t *uid;
};

struct OutDev {
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
};

// Shared-memory layout of one docking CTA: a part shared by the CTA (the
// ligand being docked) and one region per warp (one restart at a time).
struct Layout {
    int nmax, rmax, P, W, want_pose;
    // CTA part (byte offsets from the start of dynamic shared memory)
    int o_dv, o_wE, o_d0, o_wq, o_par, o_rch, o_rend, o_wR, cta_bytes;
    // warp part (byte offsets from the warp's base)
    int o_bundle, o_axis, o_X, o_best, o_tcur, o_tbest, warp_bytes;
    int total;
};

__host__ __device__ inline int lg_align16(int v) { return (v + 15) & ~15; }

__host__ __device__ inline Layout make_layout(int nmax, int rmax, int P, int W, int want_pose) {
    Layout L;
    nmax = (nmax + 3) & ~3;
    if (rmax < 1) rmax = 1;
    L.nmax = nmax; L.rmax = rmax; L.P = P; L.W = W; L.want_pose = want_pose;
    int o = 0;
    L.o_dv = o;   o = lg_align16(o + 16 * rmax);           // float4 bond vectors (grid units)
    L.o_wE = o;   o = lg_align16(o + 8 * W);               // double per warp
    L.o_d0 = o;   o = lg_align16(o + 12 * nmax);           // float x3 SoA, centroid-relative (grid units)
    L.o_wq = o;   o = lg_align16(o + 8 * nmax);            // float2 (type weight, charge)
    L.o_par = o;  o = lg_align16(o + 4 * nmax);            // int parent
    L.o_rch = o;  o = lg_align16(o + 4 * rmax);            // int torsional child
    L.o_rend = o; o = lg_align16(o + 4 * rmax);            // int end of the child's subtree
    L.o_wR = o;   o = lg_align16(o + 4 * W);               // int per warp
    L.cta_bytes = o;
    int w = 0;
    L.o_bundle = w; w = lg_align16(w + 32 * 64);           // 32 atoms x 4 float4 circle parameters
    L.o_axis = w;   w = lg_align16(w + 16 * rmax);         // float4 current bond axes
    L.o_X = w;      w = lg_align16(w + 12 * nmax);         // float x3 SoA positions
    L.o_best = w;   w = lg_align16(w + (want_pose ? 12 * nmax : 0));
    L.o_tcur = w;   w = lg_align16(w + P * rmax);
    L.o_tbest = w;  w = lg_align16(w + P * rmax);
    L.warp_bytes = w;
    L.total = L.cta_bytes + W * L.warp_bytes;
    return L;
}

// Restart-tiled warps (batched kernel): a warp docks several restarts of one
// ligand at once, kLanesPerRestart lanes per restart by default (8 restart
// slots, 9 of the 36 torsion steps per lane); the batched kernel also comes
// with 2, 8 and 16 lanes per restart (16, 4 and 2 slots).  The flattening
// kernel uses the same 4-lane step groups.
constexpr int kTile = 8;          // restarts per warp tile at 4 lanes per restart
constexpr int kLanesPerRestart = 4;
constexpr int kStepsPerLane = 9;  // 36 / 4
#ifndef LG_RT_POOL
#define LG_RT_POOL 96
#endif
constexpr int kPoolCap = LG_RT_POOL;  // flagged clash pairs buffered per warp (all its restarts)

// Per-warp shared memory of a restart-tiled warp.
struct LayoutRT {
    int o_axis, o_X, o_pool, o_mask, o_near, o_best, o_tcur, o_tbest, warp_bytes;
    int near_stride;  // bytes between the restart slots' near lists: an odd number of 4-byte words, so
                      // the slots' entries fall in different banks
};

__host__ __device__ inline LayoutRT make_layout_rt(int nmax, int rmax, int P, int want_pose, int slots = kTile) {
    LayoutRT L;
    nmax = (nmax + 3) & ~3;
    if (rmax < 1) rmax = 1;
    L.near_stride = ((nmax / 4) & 1) ? nmax : nmax + 4;
    int w = 0;
    L.o_axis = w;  w = lg_align16(w + 16 * rmax * slots);            // float4 [rmax][slots]
    L.o_X = w;     w = lg_align16(w + 12 * nmax * slots);            // float [3][nmax][slots]
    L.o_pool = w;  w = lg_align16(w + 16 * kPoolCap);                // float4 (C, A2, B2, restart slot)
    L.o_mask = w;  w = lg_align16(w + 4 * 32);                       // uint32 clash bits per lane
    L.o_near = w;  w = lg_align16(w + L.near_stride * slots);        // uint8 [slots][near_stride] near fixed atoms
    L.o_best = w;  w = lg_align16(w + (want_pose ? 12 * nmax : 0));  // float [3][nmax]
    L.o_tcur = w;  w = lg_align16(w + P * rmax * slots);             // uint8 [P*rmax][slots]
    L.o_tbest = w; w = lg_align16(w + P * rmax);                     // uint8 [P*rmax]
    L.warp_bytes = w;
    return L;
}

// Per-launch scratch (device memory beyond the inputs and outputs).
struct Scratch {
    int32_t *hist;         // kSortBuckets counters, then the work counter
    int32_t *keys;         // [L] cost bucket
    int32_t *order;        // [L] visiting order
    double *centroid;      // [3L]
    int16_t *rot_end;      // [L * rmax_lim] end of each torsional child's subtree
    // pose ranking: per CTA slot, every restart's final pose (centred grid
    // units, [S][nmax][3]), score and decisions ([S][P*rmax])
    float *rk_pose;
    double *rk_E;
    uint8_t *rk_tors;
    float *rk_G;           // [slots][S] geometric score of each restart's final pose
    float *rk_cen;         // [slots][S][3] its centroid (centred grid units)
    int rk_slots;          // ranking slots
    size_t rk_floats;      // capacity of rk_pose (floats)
    int per_cta;           // 1: centroid and rot_end hold one entry per CTA (the serving loop), not per ligand
};

// Ranking step: row p of the "within the RMSD threshold" bit matrix holds
// one bit per earlier position q < p, packed in ceil(p/32) words; rank_row_off
// is the word offset of row p (the sum of ceil(i/32) over i < p).
__host__ __device__ inline int rank_row_off(int p) {
    const int n = p - 1;
    if (n <= 0) return 0;
    const int k = (n + 31) / 32;
    return 16 * k * (k - 1) + k * (n - 32 * (k - 1));
}

// Shared memory the ranking step needs (it reuses the warps' regions):
// geometric scores and centroids (FP64), order, leaders, ranking, bit matrix.
__host__ __device__ inline int rank_smem_bytes(int S) {
    return lg_align16(8 * S) + lg_align16(24 * S) + 3 * lg_align16(4 * S) + lg_align16(4 * (rank_row_off(S) + 1)) + 64;
}

struct DockArgs {
    PocketDev pocket;
    BatchDev batch;
    OutDev out;
    Layout ly;      // CTA part (both kernels) and the plain kernel's warp part
    LayoutRT lrt;   // warp part of the restart-tiled kernel
    Scratch scr;
    int S, P;
    uint32_t seed_lo, seed_hi;
    float dc2g;                // d_clash^2 in grid units
    int nmax_lim, rmax_lim;    // per-ligand maxima (declared and within the layout)
    int rigid_steps;           // rigid greedy moves after each torsion pass
    float rigid_shift_g;       // their translation step in grid units
    int ranking;               // pose ranking on
    float thr2g;               // cluster RMSD^2 in grid units
    int rescore_top;           // K (0 = all)
    const int32_t *order;      // batched mode: ligand visiting order (NULL = identity)
    int32_t *work_counter;     // batched mode: next item of the persistent loop
    const int32_t *cls_off;    // batched mode: class boundaries in `order` (NULL = the whole batch)
    int cls;                   // with cls_off: the size class this launch docks
    int item_cap;              // > 0: dock only item_cap items evenly spread over the range (autotuning trials)
    int sort_classes;          // preparation: 1 = size class major, then cost; 0 = cost only
    int lanes;                 // batched kernel: lanes per restart of the warps' tile (2, 4, 8 or 16)
    // L2 access-policy window of the launch (host side only: the docking
    // launches carry it as a launch attribute; l2_bytes = 0: none)
    const void *l2_base;
    size_t l2_bytes;
    float l2_hit;
};

// Cost order of the batched kernels: ligands are filed by size class (atoms
// <= 32, <= 64, more) and, within a class, by estimated cost (2 buckets per
// octave); the sort visits the largest class first, costliest first.
constexpr int kCostBuckets = 64;
constexpr int kSizeClasses = 3;
constexpr int kSortBuckets = kSizeClasses * kCostBuckets;
// scratch ints after the histogram: one work counter per launch unit (each
// size class, then the whole batch) and the class boundaries in the order
// (start of class 2, class 1, class 0, then L)
constexpr int kHistInts = kSortBuckets + 2 * (kSizeClasses + 1);
__host__ __device__ inline int size_class(int n) { return n <= 32 ? 0 : (n <= 64 ? 1 : 2); }
__host__ __device__ inline int class_bound(int c) { return c == 0 ? 32 : (c == 1 ? 64 : LG_MAX_ATOMS); }

// Ligand flattening (one warp per ligand; see k_flatten).
struct FlatArgs {
    BatchDev batch;
    const int16_t *rot_end;   // from the preparation kernel, [L * rmax_lim]
    const double *centroid;   // [3L]
    int rmax_lim;
    int P;                    // passes
    float dc2;                // d_clash^2 (A^2)
    int nmax;                 // atoms per warp region (multiple of 4)
    float *xyz;               // [3A] output
    uint8_t *tors;            // [P * rot_off] output (optional)
    double *dsum;             // [L] output (optional)
    const int32_t *status;    // [L] from the preparation kernel
};

constexpr int kFlatWarps = 4;
constexpr int kFlatChunk = 128;  // pair coefficients built per round (4 per lane)
__host__ __device__ inline int flat_warp_bytes(int nmax) {
    return lg_align16(12 * nmax) + lg_align16(4 * nmax) + lg_align16(48 * nmax) + kFlatChunk * 16;
}

// Several pockets in one persistent launch: work items are (pocket, ligand)
// pairs.  pocket_major = 1 visits every ligand against pocket 0, then pocket 1,
// ... (one pocket's grids in L2 at a time); 0 gives a CTA one ligand and docks
// it against every pocket in turn.
// Passed by value (kernel parameter space): the hot loops read the pocket
// through the same constant path as the single-pocket kernel.
struct MultiDev {
    int np;
    int pocket_major;
    PocketDev pk[LG_MAX_MULTI_POCKETS];
    OutDev out[LG_MAX_MULTI_POCKETS];  // out[0] receives the preparation's status
    // per-ligand mode (merged serving requests aimed at different pockets):
    // ligand l is docked once, against pk[lig_pocket[l]], into the launch's
    // own outputs; `out` is unused
    const int32_t *lig_pocket;
};

// Device-resident serving loop (k_serve_loop): one persistent launch docks
// the ligands of admitted requests.  Each request's ligands are copied into a
// ring arena of CSR arrays in device memory (offsets global to the arena, one
// spare entry after each request), and its outputs land in an arena of mapped
// pinned host memory with the same indexing, so the launch's arguments name
// the arenas once and every ligand is a slot of them; pockets come from a
// table in the launch's arguments.  Work items are ligands numbered in
// admission order; a ring of request descriptors in device memory maps an
// item to its arena slot and pocket.  The host publishes items by raising
// `tail` (copies on a feed stream, after the data and the descriptor), a CTA
// claims the next item by fetch-and-add on `next` (one atomic per ligand,
// whatever the contention) and docks it once it is published; the CTA that
// finishes a request's last ligand raises the request's completion flag in
// mapped host memory.  A CTA that leaves while holding an unpublished item
// records it in held[CTA], and the same CTA of the next launch docks it
// first.  Every wait of the kernel is bounded (see k_serve_loop).
constexpr uint64_t kDescBusy = ~0ull;  // seq of a descriptor being rewritten
constexpr int kLoopPockets = LG_MAX_MULTI_POCKETS;

struct LoopDesc {       // one admitted request; `seq` first (seqlock: kDescBusy while rewritten)
    uint64_t seq;
    uint64_t first;     // global index of its first ligand
    int32_t L;          // its ligands
    int32_t slot;       // arena slot of its first ligand
    int32_t pocket;     // its pocket in the launch's table
    int32_t pad;
};

struct LoopCtl {        // device memory
    // written by the host (copies on the feed stream)
    uint64_t tail;      // ligands published
    uint64_t head_seq;  // descriptors before it are complete
    uint32_t stop;      // leave the loop after the current ligand
    uint32_t pad0;
    // written by the kernel
    uint64_t next;      // next ligand to claim
    uint32_t live;      // CTAs inside the loop
    uint32_t idle_exits;  // CTAs that left after the idle limit
    uint32_t bad;       // a claimed ligand had no descriptor
    uint32_t closing;   // a CTA reached the idle limit: the others leave instead of claiming
    int32_t status;     // how the launch ended: LG_OK (stopped), LG_ETIMEOUT (idle limit), LG_EINVAL (bad item)
};

struct LoopArgs {
    LoopCtl *ctl;
    const LoopDesc *desc;    // [ring]
    uint32_t *done;          // [ring] ligands finished per descriptor (reset by the last)
    uint64_t *flags;         // [ring] mapped host memory: seq + 1 once the descriptor is complete
    long long *held;         // [held_n] items CTAs claimed but left without docking (-1: none)
    int held_n;              // at least the grid of every launch of the loop
    int ring;
    uint64_t idle_ns;        // idle limit of a CTA (no ligand to claim)
    uint64_t first_seq;      // descriptors before it were complete at launch
    int np;                  // pockets in the table
    PocketDev pk[kLoopPockets];
    float dc2g[kLoopPockets], thr2g[kLoopPockets], rigid_shift_g[kLoopPockets];  // per pocket, grid units
};

// Byte size of the scratch of a launch, and its carving.
size_t scratch_bytes(int L, int rmax, int rank_slots = 0, int S = 0, int P = 0, int nmax = 0);
Scratch carve_scratch(void *base, int L, int rmax, int rank_slots = 0, int S = 0, int P = 0, int nmax = 0);

// Launchers (lg_kernels.cu)
void set_angle_tables(const float *cosv, const float *sinv);
cudaError_t launch_prep(const DockArgs &a, bool sort, cudaStream_t s, int *launches);
cudaError_t launch_fp32_peak(float *out, int blocks, int iters, cudaStream_t s);
cudaError_t launch_pack_cells(const float *go, const float *gv, const float *ge, int n, float4 *cell_o, float4 *cell_ve,
                              int num_sms, cudaStream_t s);
cudaError_t launch_dock_plain(const DockArgs &a, int ligand, int slot, cudaStream_t s);
cudaError_t launch_dock_batched(const DockArgs &a, int grid, int smem, cudaStream_t s);
cudaError_t launch_score_poses(const PocketDev &p, int L, const int32_t *atom_off, const float *xyz,
                               const float *q, const uint8_t *type, double *E, cudaStream_t s);
cudaError_t launch_diag_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int use_curand,
                               cudaStream_t s);
cudaError_t launch_dock_multi(const DockArgs &a, const MultiDev &m, int grid, int smem, cudaStream_t s);
cudaError_t launch_flatten(const FlatArgs &f, int L, cudaStream_t s);
cudaError_t launch_serve_loop(const DockArgs &a, const LoopArgs &la, int grid, int smem, cudaStream_t s);
cudaError_t loop_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid, int lanes = 4);
int checks_collect(cudaStream_t s, int rec[4]);  // bounds-check record of a debug build (0 otherwise)
cudaError_t dock_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid, bool trace, int lanes = 4);
cudaError_t multi_kernel_attributes(int W, int smem, int *ctas_per_sm, bool ranking, bool rigid);
cudaError_t plain_kernel_attributes(int smem);

}  // namespace lg
