// lg_dock_multi: one ligand batch against several loaded pockets in one
// persistent launch (the screening campaign's access pattern: a library
// against every binding site).  The preparation (validation, subtree ends,
// centroids, cost order) runs once for all pockets; work items are (pocket,
// ligand) pairs, visited pocket-major by default so one pocket's grids are in
// L2 at a time.
#include <cstring>
#include <string>
#include <vector>

#include "lg_runtime.h"

using namespace lg;

extern "C" int lg_dock_multi(lg_ctx *c, const int32_t *pocket_ids, int32_t n_pockets, const lg_ligand_batch *b,
                             const lg_dock_params *p, lg_dock_result *outs, void *stream) {
    if (!c || !pocket_ids || !b || !p || !outs) return fail(LG_EINVAL, "null argument");
    if (n_pockets < 1 || n_pockets > LG_MAX_MULTI_POCKETS) return fail(LG_EINVAL, "n_pockets out of range");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->mode != LG_MODE_BATCHED) return fail(LG_EINVAL, "lg_dock_multi runs the batched mode only");
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if (b->mem != LG_MEM_HOST && b->mem != LG_MEM_DEVICE) return fail(LG_EINVAL, "bad batch mem");
    const int32_t omem = outs[0].mem;
    for (int k = 0; k < n_pockets; k++) {
        const lg_dock_result &o = outs[k];
        if (o.mem != omem || (o.mem != LG_MEM_HOST && o.mem != LG_MEM_DEVICE))
            return fail(LG_EINVAL, "every result must have the same mem, LG_MEM_HOST or LG_MEM_DEVICE");
        if (!o.score || !o.best_restart || !o.status) return fail(LG_EINVAL, "score, best_restart and status are required");
        // optional outputs are all present or all absent, so every pocket runs the same kernel configuration
        if ((o.pose != nullptr) != (outs[0].pose != nullptr) || (o.tors_idx != nullptr) != (outs[0].tors_idx != nullptr))
            return fail(LG_EINVAL, "pose and tors_idx must be given for every pocket or for none");
    }
    if (b->L == 0) return LG_OK;
    if (!b->atom_off || !b->x || !b->y || !b->z || !b->q || !b->type || !b->parent || !b->rot_off || !b->uid)
        return fail(LG_EINVAL, "null batch array");
    std::lock_guard<std::mutex> g(c->mu);
    Range call("lg_dock_multi");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    std::vector<PocketDev> pk(n_pockets);
    for (int k = 0; k < n_pockets; k++) {
        const int pid = pocket_ids[k];
        if (pid < 0 || pid >= (int)c->pockets.size() || !c->pockets[pid].live) return fail(LG_ENOPOCKET, "unknown pocket");
        pk[k] = c->pockets[pid].dev;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int L = b->L, S = p->restarts, P = p->passes;
    int64_t A = -1, R = -1;
    int nmax, rmax;
    BatchDev bd;
    if ((rc = resolve_batch(c, b, p, s, &bd, &A, &R, &nmax, &rmax))) return rc;
    if ((int)c->multi_out.size() < n_pockets) c->multi_out.resize(n_pockets);
    std::vector<OutDev> od(n_pockets);
    for (int k = 0; k < n_pockets; k++)
        if ((rc = resolve_out(c, c->multi_out[k], b, &outs[k], S, P, p->rigid_steps, s, &A, &R, &od[k]))) return rc;
    MultiDev m;
    memset(&m, 0, sizeof(m));
    m.np = n_pockets;
    m.pocket_major = c->multi_pocket_major;
    m.lig_pocket = nullptr;
    for (int k = 0; k < n_pockets; k++) {
        m.pk[k] = pk[k];
        m.out[k] = od[k];
    }
    cudaError_t e;
    cudaEvent_t *tev = next_timing_events(c);
    if (scratch_acquire(c, s) != cudaSuccess) return fail(LG_ECUDA, "stream wait failed");
    if (m.pocket_major) {
        // pocket-major: one persistent launch per pocket, all on the preparation
        // and cost order of the first (pockets in turn keep one pocket's grids
        // in L2; measured faster than one launch over all (pocket, ligand) items)
        if (tev) cudaEventRecord(tev[0], s);
        for (int k = 0; k < n_pockets && rc == LG_OK; k++) {
            if (k > 0) {  // the preparation's per-ligand status (and the results of rejected ligands)
                e = cudaMemcpyAsync(od[k].status, od[0].status, 4 * (size_t)L, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(od[k].score, od[0].score, 8 * (size_t)L, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(od[k].best_restart, od[0].best_restart, 4 * (size_t)L,
                                        cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) {
                    rc = fail(LG_ECUDA, std::string("status copy: ") + cudaGetErrorString(e));
                    break;
                }
            }
            lg_stats st = c->stats;
            rc = dock_device(c, pk[k], bd, od[k], p, nmax, rmax, c->scratch, s, &st, nullptr, nullptr,
                             (1u << kSizeClasses) - 1, false, k > 0);
            if (k == 0) c->stats = st;
            else c->stats.launches += st.launches;
        }
        if (tev) cudaEventRecord(tev[1], s);
    } else {
        rc = dock_device(c, pk[0], bd, od[0], p, nmax, rmax, c->scratch, s, &c->stats, tev, &m);
    }
    if (scratch_release(c, s) != cudaSuccess && rc == LG_OK) rc = fail(LG_ECUDA, "event record failed");
    if (rc) return rc;
    if (omem == LG_MEM_HOST)
        for (int k = 0; k < n_pockets; k++)
            if ((rc = fetch_out(od[k], &outs[k], L, S, P, A, R, p->rigid_steps, s))) return rc;
    if (b->mem == LG_MEM_HOST || omem == LG_MEM_HOST) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("docking: ") + cudaGetErrorString(e));
    } else {
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("docking: ") + cudaGetErrorString(e));
    }
    return LG_OK;
}
