// lg_dock_batch_noalloc: batched docking that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// all device memory to their own pool allocator at start-up (an allocation
// from outside the pool would fail or fragment it), and latency-critical
// callers for whom the implicit device-wide synchronisation that
// cudaMalloc / cudaFree may perform is unacceptable.  For them this entry
// point runs the batched docking kernels with their scratch (cost buckets,
// visiting order, work counter, centroids, subtree ends) in a fixed-size
// device array that is part of the library image, instead of buffers the
// context allocates.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; each call clears the counters it needs at zero.  Calls whose work
// overlaps on the GPU (different streams, or different threads) race on the
// array: the caller must order them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "lg_runtime.h"

namespace lg {

// Scratch of lg_dock_batch_noalloc: LG_NOALLOC_SCRATCH_BYTES (4 MiB) on every
// device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LG_NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so kernels must be given this
// address.  It is looked up on every call (a host-side table lookup once the
// module is loaded), so a context re-created after cudaDeviceReset never uses
// an address of the old one; the first call on a device may load the module.
static int noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(LG_ECUDA, std::string("static scratch address: ") + cudaGetErrorString(e));
    }
    *out = p;
    return LG_OK;
}

}  // namespace lg

using namespace lg;

extern "C" int lg_dock_batch_noalloc(lg_ctx *c, int32_t pid, const lg_ligand_batch *b, const lg_dock_params *p,
                                     lg_dock_result *o, void *stream) {
    if (!c || !b || !p || !o) return fail(LG_EINVAL, "null argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->mode != LG_MODE_BATCHED) return fail(LG_EINVAL, "lg_dock_batch_noalloc runs the batched mode only");
    if (ranking_on(p)) return fail(LG_EINVAL, "lg_dock_batch_noalloc does not run pose ranking (cluster_rmsd, rescore_top)");
    if (b->mem != LG_MEM_DEVICE || o->mem != LG_MEM_DEVICE)
        return fail(LG_EINVAL, "lg_dock_batch_noalloc takes device memory only (host staging would allocate)");
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if (b->L == 0) return LG_OK;
    if (!b->atom_off || !b->x || !b->y || !b->z || !b->q || !b->type || !b->parent || !b->rot_off || !b->rot_child ||
        !b->uid)
        return fail(LG_EINVAL, "null batch array");
    if (!o->score || !o->best_restart || !o->status) return fail(LG_EINVAL, "score, best_restart and status are required");
    const int nmax = p->max_atoms > 0 ? p->max_atoms : LG_MAX_ATOMS;
    const int rmax = std::max(1, p->max_rot > 0 ? p->max_rot : LG_MAX_ROT);
    const int L = b->L;
    const size_t need = scratch_bytes(L, rmax);
    if (need > (size_t)LG_NOALLOC_SCRATCH_BYTES)
        return fail(LG_EINVAL, "batch too large for the static scratch: " + std::to_string(need) + " bytes needed, " +
                                   std::to_string((size_t)LG_NOALLOC_SCRATCH_BYTES) +
                                   " available (fewer ligands or a smaller max_rot)");

    PocketDev pk;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (pid < 0 || pid >= (int)c->pockets.size() || !c->pockets[pid].live) return fail(LG_ENOPOCKET, "unknown pocket");
        pk = c->pockets[pid].dev;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    void *base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    DockArgs a;
    memset(&a, 0, sizeof(a));
    a.pocket = pk;
    a.batch.L = L;
    a.batch.atom_off = b->atom_off;
    a.batch.x = b->x;
    a.batch.y = b->y;
    a.batch.z = b->z;
    a.batch.q = b->q;
    a.batch.type = b->type;
    a.batch.parent = b->parent;
    a.batch.rot_off = b->rot_off;
    a.batch.rot_child = b->rot_child;
    a.batch.uid = b->uid;
    a.out.score = o->score;
    a.out.best_restart = o->best_restart;
    a.out.status = o->status;
    a.out.tors_idx = o->tors_idx;
    a.out.pose = o->pose;
    a.out.restart_score = o->restart_score;
    a.out.restart_tors = o->restart_tors;
    a.out.decision_rank = o->decision_rank;
    a.out.restart_rigid = o->restart_rigid;
    a.S = p->restarts;
    a.P = p->passes;
    a.seed_lo = (uint32_t)p->seed;
    a.seed_hi = (uint32_t)(p->seed >> 32);
    const double dc = p->d_clash, h = pk.h;
    a.dc2g = (float)(dc * dc / (h * h));
    a.rigid_steps = p->rigid_steps;
    a.rigid_shift_g = (float)((double)p->rigid_shift / h);
    a.nmax_lim = nmax;
    a.rmax_lim = rmax;
    a.scr = carve_scratch(base, L, rmax);
    a.lanes = kLanesPerRestart;
    const int want_pose = o->pose != nullptr;
    int W = choose_warps(a.S, 0), occ = 0, smem = 0;
    cudaError_t e;
    for (;;) {
        a.ly = make_layout(nmax, rmax, a.P, W, want_pose);
        a.lrt = make_layout_rt(nmax, rmax, a.P, want_pose);
        smem = a.ly.cta_bytes + W * a.lrt.warp_bytes;
        if ((e = dock_kernel_attributes(W, smem, &occ, false, a.rigid_steps > 0, a.out.decision_rank != nullptr)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("dock kernel attributes: ") + cudaGetErrorString(e));
        if (occ > 0 || W == 1) break;
        W = std::max(1, W / 2);
    }
    if (occ <= 0) return fail(LG_EINVAL, "docking kernel does not fit on an SM");
    a.work_counter = a.scr.hist + kSortBuckets;
    a.order = a.scr.order;
    // the array keeps the previous call's contents: clear the bucket counters
    // and the work counter
    if ((e = cudaMemsetAsync(a.scr.hist, 0, 4 * kHistInts, s)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
    int launches = 0;
    if ((e = launch_prep(a, true, s, &launches)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("preparation launch: ") + cudaGetErrorString(e));
    const int grid = std::max(1, std::min(c->num_sms * occ, L));
    if ((e = launch_dock_batched(a, grid, smem, s)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("dock launch: ") + cudaGetErrorString(e));
#ifdef LG_CHECKS
    if ((rc = checks_result(s))) return rc;  // debug build: this call's bounds-check record
#endif
    return LG_OK;
}
