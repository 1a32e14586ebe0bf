// lg_flatten_batch: ligand flattening (paper Sec. 3.1, step 1) for a batch --
// the preparation kernel validates each ligand and finds its subtree ends and
// centroid, then k_flatten runs one warp per ligand.
#include <cmath>
#include <cstring>
#include <string>

#include "lg_runtime.h"

using namespace lg;

extern "C" int lg_flatten_batch(lg_ctx *c, const lg_ligand_batch *b, const lg_flatten_params *p, lg_flatten_result *o,
                                void *stream) {
    if (!c || !b || !p || !o) return fail(LG_EINVAL, "null argument");
    if (p->passes < 0 || p->passes > LG_MAX_PASSES) return fail(LG_EINVAL, "passes out of range");
    if (p->angle_steps != LG_ANGLE_STEPS) return fail(LG_EINVAL, "angle_steps must be 36");
    if (!(p->d_clash > 0.0f) || !std::isfinite(p->d_clash)) return fail(LG_EINVAL, "d_clash must be > 0");
    if (p->max_atoms < 0 || p->max_atoms > LG_MAX_ATOMS) return fail(LG_EINVAL, "max_atoms out of range");
    if (p->max_rot < 0 || p->max_rot > LG_MAX_ROT) return fail(LG_EINVAL, "max_rot out of range");
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if ((b->mem != LG_MEM_HOST && b->mem != LG_MEM_DEVICE) || (o->mem != LG_MEM_HOST && o->mem != LG_MEM_DEVICE))
        return fail(LG_EINVAL, "mem must be LG_MEM_HOST or LG_MEM_DEVICE");
    if (b->L == 0) return LG_OK;
    if (!b->atom_off || !b->x || !b->y || !b->z || !b->q || !b->type || !b->parent || !b->rot_off || !b->uid)
        return fail(LG_EINVAL, "null batch array");
    if (!o->xyz || !o->status) return fail(LG_EINVAL, "xyz and status are required");
    std::lock_guard<std::mutex> g(c->mu);
    Range call("lg_flatten_batch");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = b->L, P = p->passes;
    lg_dock_params dp;
    memset(&dp, 0, sizeof(dp));
    dp.restarts = 1;
    dp.passes = P;
    dp.max_atoms = p->max_atoms;
    dp.max_rot = p->max_rot;
    int64_t A = -1, R = -1;
    int nmax, rmax, rc;
    BatchDev bd;
    if ((rc = resolve_batch(c, b, &dp, s, &bd, &A, &R, &nmax, &rmax))) return rc;
    if (A < 0) {  // device batch: read the two totals (output sizes)
        int32_t tot[2];
        cudaError_t e = cudaMemcpyAsync(&tot[0], b->atom_off + L, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[1], b->rot_off + L, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("batch totals: ") + cudaGetErrorString(e));
        A = tot[0];
        R = tot[1];
    }
    nmax = std::max(1, nmax);
    rmax = std::max(1, rmax);
    // device outputs (staged for host results) and the preparation's unused score / restart outputs
    const bool host_out = o->mem == LG_MEM_HOST;
    Carve cv;
    const size_t o_dummy_s = cv.take(8 * (size_t)L), o_dummy_b = cv.take(4 * (size_t)L);
    const size_t o_xyz = host_out ? cv.take(12 * (size_t)std::max<int64_t>(A, 1)) : 0;
    const size_t o_t = host_out && o->tors ? cv.take((size_t)P * R + 1) : 0;
    const size_t o_d = host_out && o->dsum ? cv.take(8 * (size_t)L) : 0;
    const size_t o_st = host_out ? cv.take(4 * (size_t)L) : 0;
    if (c->flat_buf.ensure(cv.off)) return fail(LG_ENOMEM, "flattening buffer allocation failed");
    char *fb = (char *)c->flat_buf.p;
    float *xyz = host_out ? (float *)(fb + o_xyz) : o->xyz;
    uint8_t *tors = host_out ? (o->tors ? (uint8_t *)(fb + o_t) : nullptr) : o->tors;
    double *dsum = host_out ? (o->dsum ? (double *)(fb + o_d) : nullptr) : o->dsum;
    int32_t *status = host_out ? (int32_t *)(fb + o_st) : o->status;
    if (c->scratch.ensure(scratch_bytes(L, rmax))) return fail(LG_ENOMEM, "scratch allocation failed");
    DockArgs a;
    memset(&a, 0, sizeof(a));
    a.batch = bd;
    a.out.status = status;
    a.out.score = (double *)(fb + o_dummy_s);
    a.out.best_restart = (int32_t *)(fb + o_dummy_b);
    a.S = 1;
    a.P = P;
    a.nmax_lim = std::min(nmax, p->max_atoms > 0 ? p->max_atoms : LG_MAX_ATOMS);
    a.rmax_lim = rmax;
    a.scr = carve_scratch(c->scratch.p, L, rmax);
    int launches = 0;
    if (scratch_acquire(c, s) != cudaSuccess) return fail(LG_ECUDA, "stream wait failed");
    cudaError_t e = launch_prep(a, false, s, &launches);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("preparation launch: ") + cudaGetErrorString(e));
    FlatArgs f;
    memset(&f, 0, sizeof(f));
    f.batch = bd;
    f.rot_end = a.scr.rot_end;
    f.centroid = a.scr.centroid;
    f.rmax_lim = rmax;
    f.P = P;
    f.dc2 = p->d_clash * p->d_clash;
    f.nmax = (a.nmax_lim + 3) & ~3;
    f.xyz = xyz;
    f.tors = tors;
    f.dsum = dsum;
    f.status = status;
    e = launch_flatten(f, L, s);
    const cudaError_t er = scratch_release(c, s);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("flattening launch: ") + cudaGetErrorString(e));
    if (er != cudaSuccess) return fail(LG_ECUDA, "event record failed");
#ifdef LG_CHECKS
    if (int rc = checks_result(s)) return rc;
#endif
    if (host_out) {
        auto cp = [&](void *dst, const void *src, size_t n) {
            if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s);
        };
        cp(o->xyz, xyz, 12 * (size_t)A);
        if (o->tors) cp(o->tors, tors, (size_t)P * R);
        if (o->dsum) cp(o->dsum, dsum, 8 * (size_t)L);
        cp(o->status, status, 4 * (size_t)L);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("result download: ") + cudaGetErrorString(e));
    }
    if (b->mem == LG_MEM_HOST || host_out) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("flattening: ") + cudaGetErrorString(e));
    } else if ((e = cudaGetLastError()) != cudaSuccess) {
        return fail(LG_ECUDA, std::string("flattening: ") + cudaGetErrorString(e));
    }
    return LG_OK;
}
