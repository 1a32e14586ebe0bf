// C-ABI runtime of liblgdock (include/lg.h): contexts, pocket registry and
// cell packing, host<->device staging, launch configuration of the docking
// kernels, and the serving loop (lg_serve.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lg_internal.h"
#include "lg_runtime.h"

using namespace lg;

namespace lg {

thread_local std::string t_err;

int fail(int code, const std::string &msg) {
    t_err = msg;
    return code;
}

int DevBuf::ensure(size_t n) {
    if (n <= cap) return 0;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    cap = n;
    return 0;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}


// Pose ranking replaces the plain lowest-score choice when poses are
// clustered or only the first K ranked poses are rescored.
bool ranking_on(const lg_dock_params *p) {
    return p->cluster_rmsd > 0.0f || (p->rescore_top > 0 && p->rescore_top < p->restarts);
}

int check_params(const lg_dock_params *p) {
    if (p->restarts < 1 || p->restarts > LG_MAX_RESTARTS) return fail(LG_EINVAL, "restarts out of range");
    if (p->passes < 0 || p->passes > LG_MAX_PASSES) return fail(LG_EINVAL, "passes out of range");
    if (p->angle_steps != LG_ANGLE_STEPS) return fail(LG_EINVAL, "angle_steps must be 36");
    if (!(p->d_clash > 0.0f) || !std::isfinite(p->d_clash)) return fail(LG_EINVAL, "d_clash must be > 0");
    if (p->mode != LG_MODE_BATCHED && p->mode != LG_MODE_PLAIN) return fail(LG_EINVAL, "unknown mode");
    if (p->plain_streams < 0 || p->plain_streams > 64) return fail(LG_EINVAL, "plain_streams out of range");
    if (p->max_atoms < 0 || p->max_atoms > LG_MAX_ATOMS) return fail(LG_EINVAL, "max_atoms out of range");
    if (p->max_rot < 0 || p->max_rot > LG_MAX_ROT) return fail(LG_EINVAL, "max_rot out of range");
    if (!(p->cluster_rmsd >= 0.0f) || !std::isfinite(p->cluster_rmsd))
        return fail(LG_EINVAL, "cluster_rmsd must be finite and >= 0");
    if (p->rescore_top < 0) return fail(LG_EINVAL, "rescore_top must be >= 0");
    if (p->rigid_steps < 0 || p->rigid_steps > LG_MAX_RIGID_STEPS) return fail(LG_EINVAL, "rigid_steps out of range");
    if (!(p->rigid_shift >= 0.0f) || !std::isfinite(p->rigid_shift))
        return fail(LG_EINVAL, "rigid_shift must be finite and >= 0");
    return LG_OK;
}

// Host-side view of a batch's CSR structure (host batches only).
int host_batch_shape(const lg_ligand_batch *b, int64_t *A, int64_t *R, int *nmax, int *rmax) {
    const int L = b->L;
    if (b->atom_off[0] != 0 || b->rot_off[0] != 0) return fail(LG_EINVAL, "atom_off[0] and rot_off[0] must be 0");
    int nm = 0, rm = 0;
    for (int l = 0; l < L; l++) {
        const int64_t n = (int64_t)b->atom_off[l + 1] - b->atom_off[l];
        const int64_t r = (int64_t)b->rot_off[l + 1] - b->rot_off[l];
        if (n < 0 || r < 0) return fail(LG_EINVAL, "atom_off / rot_off must be non-decreasing");
        nm = (int)std::max<int64_t>(nm, n);
        rm = (int)std::max<int64_t>(rm, r);
    }
    *A = b->atom_off[L];
    *R = b->rot_off[L];
    *nmax = nm;
    *rmax = rm;
    return LG_OK;
}

size_t batch_image_bytes(int L, int64_t A, int64_t R) { return BatchImage(L, A, R).bytes; }

// Stage a host batch into device buffer `buf`; fills `d` with device pointers.
int stage_batch(DevBuf &buf, const lg_ligand_batch *b, int64_t A, int64_t R, BatchDev *d, cudaStream_t s) {
    if (buf.ensure(batch_image_bytes(b->L, A, R))) return fail(LG_ENOMEM, "device staging allocation failed");
    return upload_batch(buf.p, b, A, R, d, s);
}

// Copy a host batch into device memory at `dev` (batch_image_bytes bytes,
// 256-byte aligned); fills `d` with device pointers.
int upload_batch(void *dev, const lg_ligand_batch *b, int64_t A, int64_t R, BatchDev *d, cudaStream_t s) {
    const int L = b->L;
    const BatchImage im(L, A, R);
    const size_t o_aoff = im.o_aoff, o_roff = im.o_roff, o_uid = im.o_uid, o_x = im.o_x, o_y = im.o_y, o_z = im.o_z,
                 o_q = im.o_q, o_t = im.o_t, o_p = im.o_p, o_rc = im.o_rc;
    char *base = (char *)dev;
    auto cp = [&](size_t off, const void *src, size_t n) -> cudaError_t {
        if (n == 0) return cudaSuccess;
        return cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : cp(o_aoff, b->atom_off, 4 * (size_t)(L + 1));
    e = e ? e : cp(o_roff, b->rot_off, 4 * (size_t)(L + 1));
    e = e ? e : cp(o_uid, b->uid, 8 * (size_t)L);
    e = e ? e : cp(o_x, b->x, 4 * (size_t)A);
    e = e ? e : cp(o_y, b->y, 4 * (size_t)A);
    e = e ? e : cp(o_z, b->z, 4 * (size_t)A);
    e = e ? e : cp(o_q, b->q, 4 * (size_t)A);
    e = e ? e : cp(o_t, b->type, (size_t)A);
    e = e ? e : cp(o_p, b->parent, 2 * (size_t)A);
    if (R > 0) e = e ? e : cp(o_rc, b->rot_child, 2 * (size_t)R);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    d->L = L;
    d->atom_off = (const int32_t *)(base + o_aoff);
    d->rot_off = (const int32_t *)(base + o_roff);
    d->uid = (const uint64_t *)(base + o_uid);
    d->x = (const float *)(base + o_x);
    d->y = (const float *)(base + o_y);
    d->z = (const float *)(base + o_z);
    d->q = (const float *)(base + o_q);
    d->type = (const uint8_t *)(base + o_t);
    d->parent = (const int16_t *)(base + o_p);
    d->rot_child = (const int16_t *)(base + o_rc);
    return LG_OK;
}

// Device output buffers for a host result; fills `d`.
int stage_out(DevBuf &buf, const lg_dock_result *o, int L, int S, int P, int64_t A, int64_t R, int Rs, OutDev *d) {
    Carve c;
    const size_t o_s = c.take(8 * (size_t)L), o_b = c.take(4 * (size_t)L), o_st = c.take(4 * (size_t)L);
    const size_t o_t = o->tors_idx ? c.take((size_t)P * R + 1) : 0;
    const size_t o_p = o->pose ? c.take(12 * (size_t)A) : 0;
    const size_t o_rs = o->restart_score ? c.take(8 * (size_t)L * S) : 0;
    const size_t o_rt = o->restart_tors ? c.take((size_t)S * P * R + 1) : 0;
    const size_t o_rk = o->rank ? c.take(4 * (size_t)L * S) : 0;
    const size_t o_ld = o->leader ? c.take(4 * (size_t)L * S) : 0;
    const size_t o_g = o->restart_geo ? c.take(8 * (size_t)L * S) : 0;
    const size_t n_rig = (size_t)L * S * P * Rs;
    const size_t o_rg = o->restart_rigid ? c.take(n_rig + 1) : 0;
    const size_t o_dr = o->decision_rank ? c.take((size_t)S * P * R + 1) : 0;
    if (buf.ensure(c.off)) return fail(LG_ENOMEM, "device output allocation failed");
    char *base = (char *)buf.p;
    d->score = (double *)(base + o_s);
    d->best_restart = (int32_t *)(base + o_b);
    d->status = (int32_t *)(base + o_st);
    d->tors_idx = o->tors_idx ? (uint8_t *)(base + o_t) : nullptr;
    d->pose = o->pose ? (float *)(base + o_p) : nullptr;
    d->restart_score = o->restart_score ? (double *)(base + o_rs) : nullptr;
    d->restart_tors = o->restart_tors ? (uint8_t *)(base + o_rt) : nullptr;
    d->rank = o->rank ? (int32_t *)(base + o_rk) : nullptr;
    d->leader = o->leader ? (int32_t *)(base + o_ld) : nullptr;
    d->restart_geo = o->restart_geo ? (double *)(base + o_g) : nullptr;
    d->restart_rigid = o->restart_rigid ? (uint8_t *)(base + o_rg) : nullptr;
    d->decision_rank = o->decision_rank ? (uint8_t *)(base + o_dr) : nullptr;
    return LG_OK;
}

int fetch_out(const OutDev &d, const lg_dock_result *o, int L, int S, int P, int64_t A, int64_t R, int Rs,
              cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s);
    };
    cp(o->score, d.score, 8 * (size_t)L);
    cp(o->best_restart, d.best_restart, 4 * (size_t)L);
    cp(o->status, d.status, 4 * (size_t)L);
    if (o->tors_idx) cp(o->tors_idx, d.tors_idx, (size_t)P * R);
    if (o->pose) cp(o->pose, d.pose, 12 * (size_t)A);
    if (o->restart_score) cp(o->restart_score, d.restart_score, 8 * (size_t)L * S);
    if (o->restart_tors) cp(o->restart_tors, d.restart_tors, (size_t)S * P * R);
    if (o->rank) cp(o->rank, d.rank, 4 * (size_t)L * S);
    if (o->leader) cp(o->leader, d.leader, 4 * (size_t)L * S);
    if (o->restart_geo) cp(o->restart_geo, d.restart_geo, 8 * (size_t)L * S);
    if (o->restart_rigid) cp(o->restart_rigid, d.restart_rigid, (size_t)L * S * P * Rs);
    if (o->decision_rank) cp(o->decision_rank, d.decision_rank, (size_t)S * P * R);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("result download: ") + cudaGetErrorString(e));
    return LG_OK;
}

// Warps per CTA the batched kernel's launch bounds allow for a restart tile.
static int max_warps_of(int lanes) { return lanes > 4 ? lanes : 4; }

// Warps per CTA for the batched kernel: restart tiles (32 / lanes slots each)
// are spread over the CTA's warps; up to 4 warps, dividing the tile count
// when possible, unless the context option fixes the count.
int choose_warps(int S, int opt, int lanes) {
    const int slots = 32 / lanes, tiles = (S + slots - 1) / slots;
    if (opt > 0) return std::min(opt, max_warps_of(lanes));
    for (int w = std::min(tiles, 4); w >= 1; --w)
        if (tiles % w == 0) return w;
    return 1;
}

// Launch the docking of a device-resident batch on stream s: the preparation
// kernel (validation, subtree ends, centroids; cost sort in batched mode),
// then the persistent docking kernel or one plain launch per ligand.
// Size classes present in a host batch (bit c: class c).
unsigned host_class_mask(const lg_ligand_batch *b) {
    unsigned m = 0;
    for (int l = 0; l < b->L; l++) m |= 1u << size_class(std::max(1, b->atom_off[l + 1] - b->atom_off[l]));
    return m;
}

// Lanes per restart of a batch that fits in one wave, in order of preference
// (the first whose CTAs, with every restart of a ligand in flight, fit).
static const int kSmallBatchLanes[3] = {16, 8, 4};

// Restart tile (lanes per restart) and warps per CTA of a batched launch
// unit: the context options, else the autotuner's cached choice, else 4 lanes
// per restart and the restart-tile heuristic.  tiles_ok: the unit's kernel
// comes with every tile (else 4 lanes per restart).
static std::pair<int, int> tuned_tile(lg_ctx *c, const std::array<int, 8> &key, int S, bool tiles_ok, bool *cached) {
    *cached = false;
    const int wopt = c->warps_opt.load(), lopt = tiles_ok ? c->lanes_opt.load() : 0;
    const int lanes = lopt > 0 ? lopt : kLanesPerRestart;
    if (wopt > 0) {
        *cached = true;
        return {lanes, std::min(wopt, max_warps_of(lanes))};
    }
    std::lock_guard<std::mutex> g(c->tune_mu);
    auto it = c->tune.find(key);
    if (it != c->tune.end() && (tiles_ok || it->second.first == kLanesPerRestart) && (lopt == 0 || it->second.first == lopt)) {
        *cached = true;
        return it->second;
    }
    return {lanes, choose_warps(S, 0, lanes)};
}

static int dock_device_launch(lg_ctx *ctx, const PocketDev &pk, const BatchDev &bd, const OutDev &od,
                              const lg_dock_params *p, int nmax, int rmax, DevBuf &scratch, cudaStream_t s, lg_stats *st,
                              cudaEvent_t *tev, const MultiDev *multi, unsigned class_mask, bool allow_graph,
                              bool reuse_prep);

// A bounds-check record (debug builds) as the error of the call.
int checks_result(cudaStream_t s) {
    int rec[4];
    if (checks_collect(s, rec) == 0) return LG_OK;
    return fail(LG_ECUDA, "bounds check failed " + std::to_string(rec[3]) + " times; first at site " +
                              std::to_string(rec[0]) + ": index " + std::to_string(rec[1]) + " outside [0, " +
                              std::to_string(rec[2]) + ")");
}

int dock_device(lg_ctx *ctx, const PocketDev &pk, const BatchDev &bd, const OutDev &od, const lg_dock_params *p,
                int nmax, int rmax, DevBuf &scratch, cudaStream_t s, lg_stats *st, cudaEvent_t *tev,
                const MultiDev *multi, unsigned class_mask, bool allow_graph, bool reuse_prep) {
    int rc = dock_device_launch(ctx, pk, bd, od, p, nmax, rmax, scratch, s, st, tev, multi, class_mask, allow_graph,
                                reuse_prep);
#ifdef LG_CHECKS
    if (rc == LG_OK) rc = checks_result(s);
#endif
    return rc;
}

// The launch arguments of a call as key bytes, field by field (structure
// padding carries no meaning and is left out).
struct KeyBytes {
    std::vector<char> b;
    template <typename T>
    void put(const T &v) {
        const char *q = reinterpret_cast<const char *>(&v);
        b.insert(b.end(), q, q + sizeof(T));
    }
};

static void put_args(KeyBytes &k, const DockArgs &a) {
    const PocketDev &pk = a.pocket;
    k.put(pk.n), k.put(pk.h), k.put(pk.inv_h), k.put(pk.c0), k.put(pk.gmax);
    k.put(pk.center.x), k.put(pk.center.y), k.put(pk.center.z);
    k.put(pk.cell_o), k.put(pk.cell_ve), k.put(pk.pp), k.put(pk.n_pp), k.put(pk.k_out);
    for (float w : pk.type_w) k.put(w);
    const BatchDev &bd = a.batch;
    k.put(bd.L), k.put(bd.atom_off), k.put(bd.x), k.put(bd.y), k.put(bd.z), k.put(bd.q), k.put(bd.type);
    k.put(bd.parent), k.put(bd.rot_off), k.put(bd.rot_child), k.put(bd.uid);
    const OutDev &o = a.out;
    k.put(o.score), k.put(o.best_restart), k.put(o.tors_idx), k.put(o.pose), k.put(o.status), k.put(o.restart_score);
    k.put(o.restart_tors), k.put(o.rank), k.put(o.leader), k.put(o.restart_geo), k.put(o.restart_rigid);
    k.put(o.decision_rank);
    k.put(a.ly), k.put(a.lrt);  // int fields only
    const Scratch &c = a.scr;
    k.put(c.hist), k.put(c.keys), k.put(c.order), k.put(c.centroid), k.put(c.rot_end), k.put(c.rk_pose);
    k.put(c.rk_E), k.put(c.rk_tors), k.put(c.rk_G), k.put(c.rk_cen), k.put(c.rk_slots), k.put(c.rk_floats);
    k.put(c.per_cta);
    k.put(a.S), k.put(a.P), k.put(a.seed_lo), k.put(a.seed_hi), k.put(a.dc2g), k.put(a.nmax_lim), k.put(a.rmax_lim);
    k.put(a.rigid_steps), k.put(a.rigid_shift_g), k.put(a.ranking), k.put(a.thr2g), k.put(a.rescore_top);
    k.put(a.order), k.put(a.work_counter), k.put(a.cls_off), k.put(a.cls), k.put(a.item_cap), k.put(a.sort_classes);
    k.put(a.lanes), k.put(a.l2_base), k.put(a.l2_bytes), k.put(a.l2_hit);
}

static int dock_device_launch(lg_ctx *ctx, const PocketDev &pk, const BatchDev &bd, const OutDev &od,
                              const lg_dock_params *p, int nmax, int rmax, DevBuf &scratch, cudaStream_t s, lg_stats *st,
                              cudaEvent_t *tev, const MultiDev *multi, unsigned class_mask, bool allow_graph,
                              bool reuse_prep) {
    Range range("dock: prepare, tune and launch");
    const bool timed = tev != nullptr;
    DockArgs a;
    memset(&a, 0, sizeof(a));
    a.pocket = pk;
    a.batch = bd;
    a.out = od;
    a.S = p->restarts;
    a.P = p->passes;
    a.seed_lo = (uint32_t)p->seed;
    a.seed_hi = (uint32_t)(p->seed >> 32);
    const double dc = p->d_clash, h = pk.h;
    a.dc2g = (float)(dc * dc / (h * h));
    const int nmax_decl = p->max_atoms > 0 ? p->max_atoms : LG_MAX_ATOMS;
    const int rmax_decl = p->max_rot > 0 ? p->max_rot : LG_MAX_ROT;
    nmax = std::max(1, std::min(nmax, nmax_decl));
    rmax = std::max(1, std::min(rmax, rmax_decl));
    a.nmax_lim = nmax;
    a.rmax_lim = rmax;
    const int want_pose = od.pose != nullptr;
    const lg_stats keep = *st;
    memset(st, 0, sizeof(*st));
    st->dock_calls = keep.dock_calls;
    st->dock_ms_total = keep.dock_ms_total;
    st->dock_ms = keep.dock_ms;
    st->serve_loop_status = keep.serve_loop_status;
    st->serve_loop_launches = keep.serve_loop_launches;
    st->serve_loop_items = keep.serve_loop_items;
    // one pocket per launch: its overlap cells get the L2 window (not for
    // launches that dock against several pockets at once)
    if (!multi || (multi->np == 1 && !multi->lig_pocket)) l2_window_of(ctx, pk, &a.l2_base, &a.l2_bytes, &a.l2_hit);
    st->l2_window_bytes = (int64_t)a.l2_bytes;
    st->l2_persist_bytes = (int64_t)ctx->l2_persist_set;
    const int L = bd.L;
    const bool plain = p->mode == LG_MODE_PLAIN;
    if (plain && multi) return fail(LG_EINVAL, "several pockets run in the batched mode only");
    if (multi)
        for (int k = 0; k < multi->np; ++k)
            if (multi->out[k].decision_rank)
                return fail(LG_EINVAL, "decision_rank needs one launch per pocket (the pocket-major order)");
    a.rigid_steps = p->rigid_steps;
    a.rigid_shift_g = (float)((double)p->rigid_shift / h);
    a.ranking = ranking_on(p) ? 1 : 0;
    a.thr2g = (float)((double)p->cluster_rmsd * p->cluster_rmsd / (h * h));
    a.rescore_top = p->rescore_top;
    cudaError_t e;
    int launches = 0;
    // scratch holds one ranking slot per concurrently docked ligand: one per
    // plain-mode stream, one per CTA of the persistent kernel; a slot holds S
    // poses of the largest atom maximum of the launches (size classes differ)
    int scr_nmax = 0;
    auto setup_scratch = [&](int slots) -> int {
        if (scratch.ensure(scratch_bytes(L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax)))
            return fail(LG_ENOMEM, "scratch allocation failed");
        a.scr = carve_scratch(scratch.p, L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax);
        if (!plain && (e = cudaMemsetAsync(a.scr.hist, 0, 4 * kHistInts, s)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
        // merged requests for several pockets keep their pocket-grouped order
        // (one pocket's grids in L2 at a time), so no cost sort
        const bool sort = !plain && !(multi && multi->lig_pocket);
        if ((e = launch_prep(a, sort, s, &launches)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("preparation launch: ") + cudaGetErrorString(e));
        return LG_OK;
    };
    const int rank_smem = a.ranking ? rank_smem_bytes(a.S) : 0;
    if (plain) {
        const int W = std::min(a.S, 32);
        a.ly = make_layout(nmax, rmax, a.P, W, want_pose);
        scr_nmax = a.ly.nmax;
        const int psmem = std::max(a.ly.total, a.ly.cta_bytes + rank_smem);
        if ((e = plain_kernel_attributes(psmem)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("plain kernel attributes: ") + cudaGetErrorString(e));
        const int ns = p->plain_streams > 0 ? p->plain_streams : 8;
        if (int rc = setup_scratch(ns)) return rc;
        if (ctx_plain_streams(ctx, ns)) return fail(LG_ECUDA, "plain-mode stream creation failed");
        std::vector<cudaStream_t> &ps = ctx_streams(ctx);
        cudaEvent_t fork = ctx_event(ctx, 0);
        if (timed) cudaEventRecord(tev[0], s);
        cudaEventRecord(fork, s);
        for (int i = 0; i < ns; i++) cudaStreamWaitEvent(ps[i], fork, 0);
        for (int l = 0; l < L; l++) {
            if ((e = launch_dock_plain(a, l, l % ns, ps[l % ns])) != cudaSuccess)
                return fail(LG_ECUDA, std::string("plain launch: ") + cudaGetErrorString(e));
        }
        for (int i = 0; i < ns; i++) {
            cudaEvent_t j = ctx_join_event(ctx, i);
            cudaEventRecord(j, ps[i]);
            cudaStreamWaitEvent(s, j, 0);
        }
        if (timed) cudaEventRecord(tev[1], s);
        st->launches = launches + L;
        st->grid = L;
        st->warps_per_cta = W;
        st->restart_lanes = 32;
        st->ctas_per_sm = 1;
        st->smem_bytes = psmem;
        return LG_OK;
    }
    // batched: cost-ordered persistent launches of restart-tiled warps, one
    // per size class when the batch's atom maximum exceeds 64 (each class
    // with shared memory for its own maximum, so small ligands keep a high
    // occupancy), else one for the whole batch
    struct Unit {
        int cls, nmax, W, lanes, occ, smem, grid;
        bool tuned;
        std::array<int, 8> key;
    };
    std::vector<Unit> units;
    const bool split = !multi && ctx->size_classes && nmax > class_bound(1);
    const bool trace = a.out.decision_rank != nullptr;
    // tiles other than 4 lanes per restart: the single-pocket kernel without
    // ranking or decision ranks
    const bool tiles_ok = !multi && !a.ranking && !trace;
    auto configure = [&](Unit &u) -> int {
        for (;;) {
            a.ly = make_layout(u.nmax, rmax, a.P, u.W, want_pose);
            a.lrt = make_layout_rt(u.nmax, rmax, a.P, want_pose, 32 / u.lanes);
            u.smem = std::max(a.ly.cta_bytes + u.W * a.lrt.warp_bytes, a.ly.cta_bytes + rank_smem);
            e = multi ? multi_kernel_attributes(u.W, u.smem, &u.occ, a.ranking, a.rigid_steps > 0)
                      : dock_kernel_attributes(u.W, u.smem, &u.occ, a.ranking, a.rigid_steps > 0, trace, u.lanes);
            if (e != cudaSuccess) return fail(LG_ECUDA, std::string("dock kernel attributes: ") + cudaGetErrorString(e));
            if (u.occ > 0 || u.W == 1) break;
            u.W = std::max(1, u.W / 2);
        }
        if (u.occ <= 0) return fail(LG_EINVAL, "docking kernel does not fit on an SM");
        const long items = multi && multi->pocket_major && !multi->lig_pocket ? (long)L * multi->np : (long)L;
        u.grid = (int)std::max(1L, std::min((long)ctx_num_sms(ctx) * u.occ, items));
        return LG_OK;
    };
    for (int c = kSizeClasses - 1; c >= -1; --c) {
        if (split ? (c < 0 || !((class_mask >> c) & 1u)) : c >= 0) continue;
        Unit u;
        u.cls = c;
        u.nmax = c < 0 ? nmax : std::min(nmax, class_bound(c));
        // launch kind: one pocket; several pockets ligand-major, pocket-major, or one pocket per ligand
        const int kind = !multi ? 0 : (multi->lig_pocket ? 3 : (multi->pocket_major ? 2 : 1));
        u.key = {c, a.S, a.P, u.nmax, rmax, a.ranking + 2 * (trace ? 1 : 0), a.rigid_steps > 0 ? 1 : 0, want_pose + 2 * kind};
        const std::pair<int, int> t = tuned_tile(ctx, u.key, a.S, tiles_ok, &u.tuned);
        u.lanes = t.first;
        u.W = t.second;
        if (int rc = configure(u)) return rc;
        units.push_back(u);
    }
    // A batch too small to fill the GPU gets a latency tile unless the context
    // fixes the width: when every item fits in one wave, each ligand runs in
    // one CTA with all its restarts at once, over as many lanes per restart as
    // the preference order below allows (more lanes per restart: fewer steps
    // per lane, so a shorter chain of decisions); the tuned tile is for full
    // batches and is neither used nor tuned here
    if (ctx->warps_opt.load() <= 0) {
        const long items = multi && multi->pocket_major && !multi->lig_pocket ? (long)L * multi->np : (long)L;
        const int lopt = tiles_ok ? ctx->lanes_opt.load() : 0;
        std::vector<int> prefs;
        if (lopt > 0)
            prefs = {lopt};
        else if (tiles_ok)
            prefs = {kSmallBatchLanes[0], kSmallBatchLanes[1], kSmallBatchLanes[2]};
        else
            prefs = {kLanesPerRestart};
        for (Unit &u : units)
            for (int lanes : prefs) {
                const int slots = 32 / lanes, full = std::min(max_warps_of(lanes), (a.S + slots - 1) / slots);
                Unit v = u;
                v.lanes = lanes;
                v.W = full;
                if (configure(v) == LG_OK && v.W == full && items <= (long)ctx_num_sms(ctx) * v.occ) {
                    u = v;
                    u.tuned = true;
                    break;
                }
            }
    }
    a.sort_classes = split ? 1 : 0;
    for (const Unit &u : units) scr_nmax = std::max(scr_nmax, make_layout(u.nmax, rmax, a.P, 1, want_pose).nmax);
    // autotuning candidates (lanes per restart, warps per CTA)
    std::vector<std::pair<int, int>> cands;
    {
        const int lopt = tiles_ok ? ctx->lanes_opt.load() : 0;
        if (lopt > 0)
            cands = {{lopt, 4}, {lopt, 2}, {lopt, 1}};
        else if (tiles_ok)
            cands = {{4, 4}, {4, 2}, {4, 1}, {2, 2}, {2, 1}, {8, 4}, {8, 2}};
        else
            cands = {{4, 4}, {4, 2}, {4, 1}};
    }
    int slots = 1;
    for (const Unit &u : units) slots = std::max(slots, u.grid);
    bool need_tune = false;  // tuning trials run eagerly on the sorted batch: no graph for this call
    for (const Unit &u : units) need_tune = need_tune || (ctx->autotune && !u.tuned);
    if (need_tune)  // ranking slots for every candidate's grid
        for (const Unit &u : units)
            for (const auto &c : cands) {
                Unit v = u;
                v.lanes = c.first;
                v.W = c.second;
                if (!u.tuned && configure(v) == LG_OK) slots = std::max(slots, v.grid);
            }
    // key of a call: the launch arguments, the units and the stream
    auto call_key = [&]() {
        KeyBytes k;
        put_args(k, a);
        for (const Unit &u : units) {
            const int v[7] = {u.cls, u.nmax, u.W, u.lanes, u.smem, u.grid, u.occ};
            k.put(v);
        }
        k.put(s);
        return std::move(k.b);
    };
    bool graph = allow_graph && ctx->graphs.load() > 0 && !multi && s != nullptr && !need_tune && !reuse_prep;
    if (graph && ctx->graphs.load() == 2) {  // capture only arguments seen before (the second call on)
        std::vector<char> k = call_key();
        auto &seen = ctx->graph_seen;
        if (std::find(seen.begin(), seen.end(), k) == seen.end()) {
            seen.push_back(std::move(k));
            if (seen.size() > 16) seen.erase(seen.begin());
            graph = false;
        }
    }
    if (reuse_prep) {  // the same batch was prepared and sorted by the previous call: clear the work counters
        if (scratch.ensure(scratch_bytes(L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax)))
            return fail(LG_ENOMEM, "scratch allocation failed");
        a.scr = carve_scratch(scratch.p, L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax);
        if ((e = cudaMemsetAsync(a.scr.hist + kSortBuckets, 0, 4 * (kSizeClasses + 1), s)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
    } else if (!graph) {
        if (int rc = setup_scratch(slots)) return rc;
    } else {  // the preparation goes into the graph with the docking launches
        if (scratch.ensure(scratch_bytes(L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax)))
            return fail(LG_ENOMEM, "scratch allocation failed");
        a.scr = carve_scratch(scratch.p, L, rmax, a.ranking ? slots : 0, a.S, a.P, scr_nmax);
    }
    a.order = (multi && multi->lig_pocket) ? nullptr : a.scr.order;
    int32_t *counters = a.scr.hist + kSortBuckets;
    // the kernels' shared-memory limit is per function: the largest of the
    // units that launch the same kernel (same restart tile)
    auto set_limit = [&]() -> cudaError_t {
        for (const Unit &u : units) {
            int big = 0, occ = 0;
            for (const Unit &o : units)
                if (o.lanes == u.lanes) big = std::max(big, o.smem);
            const cudaError_t r = multi ? multi_kernel_attributes(u.W, big, &occ, a.ranking, a.rigid_steps > 0)
                                        : dock_kernel_attributes(u.W, big, &occ, a.ranking, a.rigid_steps > 0, trace, u.lanes);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    auto launch_unit = [&](const Unit &u, int cap, cudaStream_t us) -> cudaError_t {
        a.ly = make_layout(u.nmax, rmax, a.P, u.W, want_pose);
        a.lrt = make_layout_rt(u.nmax, rmax, a.P, want_pose, 32 / u.lanes);
        a.lanes = u.lanes;
        a.cls = u.cls;
        a.cls_off = u.cls >= 0 ? counters + kSizeClasses + 1 : nullptr;
        a.work_counter = counters + (u.cls >= 0 ? u.cls : kSizeClasses);
        a.item_cap = cap;
        return multi ? launch_dock_multi(a, *multi, u.grid, u.smem, us) : launch_dock_batched(a, u.grid, u.smem, us);
    };
    // The units of a call: with several size classes and no pose ranking
    // (whose slots belong to CTA indices), the classes after the first run on
    // the context's class streams, forked from s and joined back into it, so
    // that one class's last wave overlaps the next class's first (each class
    // has its own work counter; outputs are per ligand)
    auto launch_units = [&]() -> cudaError_t {
        if (units.size() == 1 || a.ranking) {
            for (const Unit &u : units)
                if (cudaError_t r = launch_unit(u, 0, s)) return r;
            return cudaSuccess;
        }
        std::lock_guard<std::mutex> g(ctx->class_mu);
        if (ctx_class_streams(ctx)) return cudaErrorMemoryAllocation;
        cudaError_t r = cudaEventRecord(ctx->class_fork, s);
        for (size_t i = 0; i < units.size() && r == cudaSuccess; ++i) {
            cudaStream_t us = i == 0 ? s : ctx->class_streams[i - 1];
            if (i > 0) r = cudaStreamWaitEvent(us, ctx->class_fork, 0);
            if (r == cudaSuccess) r = launch_unit(units[i], 0, us);
        }
        for (size_t i = 1; i < units.size() && r == cudaSuccess; ++i) {
            r = cudaEventRecord(ctx->class_join[i - 1], ctx->class_streams[i - 1]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(s, ctx->class_join[i - 1], 0);
        }
        return r;
    };
    // autotuning: a unit without a cached choice times every candidate on the
    // first ligands of its class (same order, same ligands), keeps the fastest
    // and re-clears its work counter; the results do not depend on the choice
    if (ctx->autotune)
        for (Unit &u : units) {
            if (u.tuned) continue;
            // the same ligands for every candidate: an even sample of the
            // class's cost order, 16 waves of the widest candidate's grid (at
            // least 4,096)
            int cap = 4096;
            for (const auto &c : cands) {
                Unit v = u;
                v.lanes = c.first;
                v.W = c.second;
                if (configure(v) == LG_OK && v.W == c.second) cap = std::max(cap, 16 * v.grid);
            }
            float best = INFINITY;
            Unit keep = u;
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
                if (t0) cudaEventDestroy(t0);
                return fail(LG_ECUDA, std::string("autotuning events: ") + cudaGetErrorString(e));
            }
            for (const auto &c : cands) {
                Unit v = u;
                v.lanes = c.first;
                v.W = c.second;
                if (configure(v) != LG_OK || v.W != c.second) continue;
                if (v.grid > slots) continue;  // ranking slots are sized for the launches above
                if ((e = cudaMemsetAsync(counters + (u.cls >= 0 ? u.cls : kSizeClasses), 0, 4, s)) != cudaSuccess ||
                    (e = cudaEventRecord(t0, s)) != cudaSuccess || (e = launch_unit(v, cap, s)) != cudaSuccess ||
                    (e = cudaEventRecord(t1, s)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess) {
                    cudaEventDestroy(t0);
                    cudaEventDestroy(t1);
                    return fail(LG_ECUDA, std::string("autotuning: ") + cudaGetErrorString(e));
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, t0, t1);
                launches++;
                if (ms < best) {
                    best = ms;
                    keep = v;
                }
            }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            u = keep;
            {
                std::lock_guard<std::mutex> g(ctx->tune_mu);
                ctx->tune[u.key] = {u.lanes, u.W};
            }
            if ((e = cudaMemsetAsync(counters + (u.cls >= 0 ? u.cls : kSizeClasses), 0, 4, s)) != cudaSuccess)
                return fail(LG_ECUDA, std::string("autotuning: ") + cudaGetErrorString(e));
        }
    if ((e = set_limit()) != cudaSuccess)
        return fail(LG_ECUDA, std::string("dock kernel attributes: ") + cudaGetErrorString(e));
    if (graph) {
        // key: the launch arguments after carving, the units and the stream
        std::vector<char> key = call_key();
        auto &cache = ctx->graph_cache;
        int hit = -1;
        for (int i = 0; i < (int)cache.size(); i++)
            if (cache[i].key == key) hit = i;
        if (hit < 0) {
            const int before = launches;
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return fail(LG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            cudaError_t ec = cudaMemsetAsync(a.scr.hist, 0, 4 * kHistInts, s);
            if (ec == cudaSuccess) ec = launch_prep(a, true, s, &launches);
            if (ec == cudaSuccess) ec = launch_units();
            e = cudaStreamEndCapture(s, &g);
            if (ec != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return fail(LG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec != cudaSuccess ? ec : e));
            }
            lg_ctx::GraphRec rec;
            rec.key = std::move(key);
            rec.launches = launches - before + (int)units.size();
            e = cudaGraphInstantiate(&rec.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(LG_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
            if (cache.size() >= 8) {
                cudaGraphExecDestroy(cache.front().exec);
                cache.erase(cache.begin());
            }
            cache.push_back(std::move(rec));
            hit = (int)cache.size() - 1;
            st->graph = 2;
        } else {
            lg_ctx::GraphRec rec = std::move(cache[hit]);  // most recently used last
            cache.erase(cache.begin() + hit);
            cache.push_back(std::move(rec));
            hit = (int)cache.size() - 1;
            st->graph = 1;
        }
        if (timed) cudaEventRecord(tev[0], s);
        if ((e = cudaGraphLaunch(cache[hit].exec, s)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        if (timed) cudaEventRecord(tev[1], s);
        const Unit &u0 = units.front();
        st->launches = cache[hit].launches;
        st->grid = u0.grid;
        st->warps_per_cta = u0.W;
        st->restart_lanes = u0.lanes;
        st->ctas_per_sm = u0.occ;
        st->smem_bytes = u0.smem;
        return LG_OK;
    }
    if (timed) cudaEventRecord(tev[0], s);
    if ((e = launch_units()) != cudaSuccess) return fail(LG_ECUDA, std::string("dock launch: ") + cudaGetErrorString(e));
    if (timed) cudaEventRecord(tev[1], s);
    const Unit &u0 = units.front();
    st->launches = launches + (int)units.size();
    st->grid = u0.grid;
    st->warps_per_cta = u0.W;
    st->restart_lanes = u0.lanes;
    st->ctas_per_sm = u0.occ;
    st->smem_bytes = u0.smem;
    return LG_OK;
}

// Device view of a batch: staged into the context's input buffer for host
// batches (which also yields the totals and the measured maxima), as given
// for device batches.
int resolve_batch(lg_ctx *c, const lg_ligand_batch *b, const lg_dock_params *p, cudaStream_t s, BatchDev *bd,
                  int64_t *A, int64_t *R, int *nmax, int *rmax) {
    const int L = b->L;
    int rc;
    *A = -1;
    *R = -1;
    *nmax = p->max_atoms > 0 ? p->max_atoms : LG_MAX_ATOMS;
    *rmax = p->max_rot > 0 ? p->max_rot : LG_MAX_ROT;
    if (b->mem == LG_MEM_HOST) {
        int nm, rm;
        if ((rc = host_batch_shape(b, A, R, &nm, &rm))) return rc;
        if (*R > 0 && !b->rot_child) return fail(LG_EINVAL, "null rot_child");
        *nmax = std::min(*nmax, std::max(nm, 1));
        *rmax = std::min(*rmax, std::max(rm, 1));
        return stage_batch(c->in_buf, b, *A, *R, bd, s);
    }
    if (!b->rot_child) return fail(LG_EINVAL, "null rot_child");
    bd->L = L;
    bd->atom_off = b->atom_off;
    bd->x = b->x;
    bd->y = b->y;
    bd->z = b->z;
    bd->q = b->q;
    bd->type = b->type;
    bd->parent = b->parent;
    bd->rot_off = b->rot_off;
    bd->rot_child = b->rot_child;
    bd->uid = b->uid;
    return LG_OK;
}

// Device view of a result: device buffers from `buf` for host results (the
// totals of a device batch are read back first), as given for device results.
int resolve_out(lg_ctx *c, DevBuf &buf, const lg_ligand_batch *b, const lg_dock_result *o, int S, int P, int Rs,
                cudaStream_t s, int64_t *A, int64_t *R, OutDev *od) {
    (void)c;
    const int L = b->L;
    if (o->mem == LG_MEM_HOST) {
        if (*A < 0) {  // device batch, host result: read the two totals
            int32_t tot[2];
            cudaError_t e = cudaMemcpyAsync(&tot[0], b->atom_off + L, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&tot[1], b->rot_off + L, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(LG_ECUDA, std::string("batch totals: ") + cudaGetErrorString(e));
            *A = tot[0];
            *R = tot[1];
        }
        return stage_out(buf, o, L, S, P, *A, *R, Rs, od);
    }
    od->score = o->score;
    od->best_restart = o->best_restart;
    od->status = o->status;
    od->tors_idx = o->tors_idx;
    od->pose = o->pose;
    od->restart_score = o->restart_score;
    od->restart_tors = o->restart_tors;
    od->rank = o->rank;
    od->leader = o->leader;
    od->restart_geo = o->restart_geo;
    od->restart_rigid = o->restart_rigid;
    od->decision_rank = o->decision_rank;
    return LG_OK;
}

// Event pair of the next timed call (NULL when timing is off).
cudaEvent_t *next_timing_events(lg_ctx *c) {
    if (!c->timing) return nullptr;
    if (c->tev_pending == lg_ctx::kTimingRing) harvest_timing(c);
    cudaEvent_t *tev = c->tev[c->tev_head];
    c->tev_head = (c->tev_head + 1) % lg_ctx::kTimingRing;
    c->tev_pending++;
    return tev;
}

// Wait for the timed calls still in the ring and add their device times.
void harvest_timing(lg_ctx *c) {
    while (c->tev_pending > 0) {
        const int i = (c->tev_head - c->tev_pending + lg_ctx::kTimingRing) % lg_ctx::kTimingRing;
        float ms = 0.0f;
        if (cudaEventSynchronize(c->tev[i][1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, c->tev[i][0], c->tev[i][1]) == cudaSuccess) {
            c->stats.dock_ms = ms;
            c->stats.dock_ms_total += ms;
            c->stats.dock_calls++;
        } else {
            cudaGetLastError();
        }
        c->tev_pending--;
    }
}

// L2 access-policy window of a pocket's overlap cells (the lookups of every
// torsion step): the cells, capped at the device's window limit, with the
// share of them the persisting set-aside can hold as the hit ratio.
void l2_window_of(lg_ctx *c, const PocketDev &pk, const void **base, size_t *bytes, float *hit) {
    *base = nullptr;
    *bytes = 0;
    *hit = 0.0f;
    if (!c->l2_window.load() || c->l2_persist_set == 0 || c->l2_window_max == 0) return;
    const size_t n = (size_t)pk.n, cells = n * n * n * 32;
    *base = pk.cell_o;
    *bytes = std::min(cells, c->l2_window_max);
    *hit = (float)std::min(1.0, (double)c->l2_persist_set / (double)*bytes);
}

// Persisting L2 set-aside for the loaded pockets: room for the largest
// pocket's overlap cells (the pocket a launch docks against), within the
// device's maximum.  A context limit: it ends with the context.
static void l2_reserve(lg_ctx *c) {
    if (c->l2_persist_max == 0) return;
    size_t want = 0;
    for (const auto &p : c->pockets)
        if (p.live) want = std::max(want, (size_t)p.dev.n * p.dev.n * p.dev.n * 32);
    want = std::min(want, c->l2_persist_max);
    if (want == c->l2_persist_set) return;
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) {
        c->l2_persist_set = want;
    } else {
        cudaGetLastError();  // no set-aside: launches then carry no window
        c->l2_persist_set = 0;
    }
}

// Pocket packing: trilinear coefficients per node (FP64, rounded to FP32).
static void pack_cells(const float *g, int n, float *out, int stride, int offset) {
    auto at = [&](int i, int j, int k) -> double {
        i = std::min(i, n - 1);
        j = std::min(j, n - 1);
        k = std::min(k, n - 1);
        return (double)g[((size_t)k * n + j) * n + i];
    };
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                const double v000 = at(i, j, k), v100 = at(i + 1, j, k), v010 = at(i, j + 1, k),
                             v110 = at(i + 1, j + 1, k), v001 = at(i, j, k + 1), v101 = at(i + 1, j, k + 1),
                             v011 = at(i, j + 1, k + 1), v111 = at(i + 1, j + 1, k + 1);
                float *o = out + ((size_t)k * n * n + (size_t)j * n + i) * stride + offset;
                o[0] = (float)v000;
                o[1] = (float)(v100 - v000);
                o[2] = (float)(v010 - v000);
                o[3] = (float)(v001 - v000);
                o[4] = (float)(v110 - v100 - v010 + v000);
                o[5] = (float)(v101 - v100 - v001 + v000);
                o[6] = (float)(v011 - v010 - v001 + v000);
                o[7] = (float)(v111 - v110 - v101 - v011 + v100 + v010 + v001 - v000);
            }
}

}  // namespace lg

// ======================================================================= C ABI
extern "C" {

int lg_create(int device, lg_ctx **out) {
    if (!out) return fail(LG_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return fail(LG_ECUDA, "no CUDA device");
    }
    if (device < 0 || device >= count) return fail(LG_EINVAL, "device out of range");
    lg_ctx *c = new (std::nothrow) lg_ctx();
    if (!c) return fail(LG_ENOMEM, "context allocation failed");
    c->device = device;
    c->stats.serve_loop_status = -1;
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
        delete c;
        return fail(LG_ECUDA, std::string("device setup: ") + cudaGetErrorString(e));
    }
    {
        int pmax = 0, wmax = 0;
        if (cudaDeviceGetAttribute(&pmax, cudaDevAttrMaxPersistingL2CacheSize, device) == cudaSuccess &&
            cudaDeviceGetAttribute(&wmax, cudaDevAttrMaxAccessPolicyWindowSize, device) == cudaSuccess &&
            cudaDeviceGetLimit(&c->l2_persist_prev, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
            c->l2_persist_max = (size_t)std::max(pmax, 0);
            c->l2_window_max = (size_t)std::max(wmax, 0);
        } else {
            cudaGetLastError();
        }
    }
    for (int i = 0; i < 3; i++) cudaEventCreate(&c->ev[i]);
    cudaEventCreateWithFlags(&c->scratch_ev, cudaEventDisableTiming);
    for (int i = 0; i < lg_ctx::kTimingRing; i++)
        for (int j = 0; j < 2; j++) cudaEventCreate(&c->tev[i][j]);
    float cs[LG_ANGLE_STEPS], sn[LG_ANGLE_STEPS];
    for (int t = 0; t < LG_ANGLE_STEPS; t++) {
        const double th = 2.0 * M_PI * t / LG_ANGLE_STEPS;
        cs[t] = (float)cos(th);
        sn[t] = (float)sin(th);
    }
    set_angle_tables(cs, sn);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        lg_destroy(c);
        return fail(LG_ECUDA, std::string("angle tables: ") + cudaGetErrorString(e));
    }
    *out = c;
    return LG_OK;
}

void lg_destroy(lg_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    serve_stop(c);
    cudaDeviceSynchronize();
    for (auto &p : c->pockets)
        if (p.mem) cudaFree(p.mem);
    if (c->l2_persist_set) {  // lines marked persisting go back to normal; the limit found at creation
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_persist_prev);
        cudaGetLastError();
    }
    c->in_buf.release();
    c->out_buf.release();
    c->scratch.release();
    for (auto &m : c->multi_out) m.release();
    for (auto &g : c->graph_cache) cudaGraphExecDestroy(g.exec);
    c->flat_buf.release();
    for (auto s : c->plain_streams) cudaStreamDestroy(s);
    for (auto ev : c->join_events) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) {
        if (c->class_streams[i]) cudaStreamDestroy(c->class_streams[i]);
        if (c->class_join[i]) cudaEventDestroy(c->class_join[i]);
    }
    if (c->class_fork) cudaEventDestroy(c->class_fork);
    for (int i = 0; i < 3; i++)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->scratch_ev) cudaEventDestroy(c->scratch_ev);
    for (int i = 0; i < lg_ctx::kTimingRing; i++)
        for (int j = 0; j < 2; j++)
            if (c->tev[i][j]) cudaEventDestroy(c->tev[i][j]);
    delete c;
}

const char *lg_last_error(lg_ctx *) { return t_err.c_str(); }

int lg_pocket_load(lg_ctx *c, const lg_pocket_desc *d, int32_t *pid) {
    if (!c || !d || !pid) return fail(LG_EINVAL, "null argument");
    const int n = d->n;
    if (n < 2 || n > 512) return fail(LG_EINVAL, "grid size n must be in [2, 512]");
    if (!(d->h > 0.0f) || !std::isfinite(d->h)) return fail(LG_EINVAL, "h must be > 0");
    if (!d->phi_o || !d->phi_v || !d->phi_e || !d->pocket_points) return fail(LG_EINVAL, "null grid pointer");
    if (d->n_pp < 1) return fail(LG_EINVAL, "n_pp must be >= 1");
    for (int c3 = 0; c3 < 3; c3++)
        if (!std::isfinite(d->origin[c3])) return fail(LG_EINVAL, "origin must be finite");
    const size_t n3 = (size_t)n * n * n;
    for (size_t t = 0; t < n3; t++)
        if (!std::isfinite(d->phi_o[t]) || !std::isfinite(d->phi_v[t]) || !std::isfinite(d->phi_e[t]))
            return fail(LG_EINVAL, "grid values must be finite");
    for (int i = 0; i < 3 * d->n_pp; i++)
        if (d->pocket_points[i] < 0 || d->pocket_points[i] >= n) return fail(LG_EINVAL, "pocket point outside grid");
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");

    std::vector<float> h_pp(4 * (size_t)d->n_pp);
    const double c0 = (n - 1) / 2.0;
    for (int p = 0; p < d->n_pp; p++) {
        for (int c3 = 0; c3 < 3; c3++) h_pp[4 * p + c3] = (float)(d->pocket_points[3 * p + c3] - c0);
        h_pp[4 * p + 3] = 0.0f;
    }
    Carve cv;
    const size_t o_o = cv.take(n3 * 32), o_ve = cv.take(n3 * 64), o_pp = cv.take(h_pp.size() * 4);
    void *mem = nullptr;
    if (cudaMalloc(&mem, cv.off) != cudaSuccess) {
        cudaGetLastError();
        return fail(LG_ENOMEM, "pocket allocation failed");
    }
    char *base = (char *)mem;
    cudaError_t e = cudaMemcpy(base + o_pp, h_pp.data(), h_pp.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->pack_host) {  // the host packing (same arithmetic), for comparison
        std::vector<float> h_o(n3 * 8), h_ve(n3 * 16);
        pack_cells(d->phi_o, n, h_o.data(), 8, 0);
        pack_cells(d->phi_v, n, h_ve.data(), 16, 0);
        pack_cells(d->phi_e, n, h_ve.data(), 16, 8);
        e = cudaMemcpy(base + o_o, h_o.data(), h_o.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(base + o_ve, h_ve.data(), h_ve.size() * 4, cudaMemcpyHostToDevice);
    } else if (e == cudaSuccess) {
        // the three raw grids (12 B per node, an eighth of the packed cells)
        // go up once and the device packs them
        void *raw = nullptr;
        if (cudaMalloc(&raw, 12 * n3) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(mem);
            return fail(LG_ENOMEM, "pocket staging allocation failed");
        }
        float *r = (float *)raw;
        e = cudaMemcpy(r, d->phi_o, 4 * n3, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(r + n3, d->phi_v, 4 * n3, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(r + 2 * n3, d->phi_e, 4 * n3, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_pack_cells(r, r + n3, r + 2 * n3, n, (float4 *)(base + o_o), (float4 *)(base + o_ve),
                                  ctx_num_sms(c), 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        cudaFree(raw);
    }
    if (e != cudaSuccess) {
        cudaFree(mem);
        return fail(LG_ECUDA, std::string("pocket upload: ") + cudaGetErrorString(e));
    }
    PocketRec r;
    r.live = true;
    r.mem = mem;
    r.bytes = cv.off;
    PocketDev &pd = r.dev;
    pd.n = n;
    pd.h = d->h;
    pd.inv_h = (float)(1.0 / (double)d->h);
    pd.c0 = (float)c0;
    pd.gmax = (float)(n - 1);
    pd.center = make_float3((float)(d->origin[0] + d->h * c0), (float)(d->origin[1] + d->h * c0),
                            (float)(d->origin[2] + d->h * c0));
    pd.cell_o = (const float4 *)(base + o_o);
    pd.cell_ve = (const float4 *)(base + o_ve);
    pd.pp = (const float4 *)(base + o_pp);
    pd.n_pp = d->n_pp;
    for (int t = 0; t < LG_NUM_TYPES; t++) pd.type_w[t] = d->type_w[t];
    pd.k_out = d->k_out;
    int id = -1;
    for (size_t i = 0; i < c->pockets.size(); i++)
        if (!c->pockets[i].live) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)c->pockets.size();
        c->pockets.push_back(r);
    } else {
        c->pockets[id] = r;
    }
    l2_reserve(c);
    {
        std::lock_guard<std::mutex> pg(c->pk_mu);
        c->live_pockets.push_back(pd);
    }
    *pid = id;
    return LG_OK;
}

int lg_pocket_unload(lg_ctx *c, int32_t pid) {
    if (!c) return fail(LG_EINVAL, "null context");
    std::lock_guard<std::mutex> g(c->mu);
    if (pid < 0 || pid >= (int)c->pockets.size() || !c->pockets[pid].live) return fail(LG_ENOPOCKET, "unknown pocket");
    cudaSetDevice(c->device);
    {
        std::lock_guard<std::mutex> pg(c->pk_mu);
        auto &v = c->live_pockets;
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i].cell_o == c->pockets[pid].dev.cell_o) {
                v.erase(v.begin() + i);
                break;
            }
    }
    cudaFree(c->pockets[pid].mem);
    c->pockets[pid] = PocketRec();
    l2_reserve(c);
    return LG_OK;
}

int lg_dock_batch(lg_ctx *c, int32_t pid, const lg_ligand_batch *b, const lg_dock_params *p, lg_dock_result *o,
                  void *stream) {
    if (!c || !b || !p || !o) return fail(LG_EINVAL, "null argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if ((b->mem != LG_MEM_HOST && b->mem != LG_MEM_DEVICE) || (o->mem != LG_MEM_HOST && o->mem != LG_MEM_DEVICE))
        return fail(LG_EINVAL, "mem must be LG_MEM_HOST or LG_MEM_DEVICE");
    if (b->L == 0) return LG_OK;
    if (!b->atom_off || !b->x || !b->y || !b->z || !b->q || !b->type || !b->parent || !b->rot_off || !b->uid)
        return fail(LG_EINVAL, "null batch array");
    if (!o->score || !o->best_restart || !o->status) return fail(LG_EINVAL, "score, best_restart and status are required");
    std::lock_guard<std::mutex> g(c->mu);
    Range call("lg_dock_batch");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    PocketRec *pk = (pid >= 0 && pid < (int)c->pockets.size() && c->pockets[pid].live) ? &c->pockets[pid] : nullptr;
    if (!pk) return fail(LG_ENOPOCKET, "unknown pocket");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = b->L, S = p->restarts, P = p->passes;

    int64_t A = -1, R = -1;
    int nmax, rmax;
    BatchDev bd;
    OutDev od;
    {
        Range stage("stage inputs and outputs");
        if ((rc = resolve_batch(c, b, p, s, &bd, &A, &R, &nmax, &rmax))) return rc;
        if ((rc = resolve_out(c, c->out_buf, b, o, S, P, p->rigid_steps, s, &A, &R, &od))) return rc;
    }
    cudaEvent_t *tev = next_timing_events(c);
    const unsigned cmask = b->mem == LG_MEM_HOST ? host_class_mask(b) : (1u << kSizeClasses) - 1;
    const bool graph_ok = b->mem == LG_MEM_DEVICE && o->mem == LG_MEM_DEVICE;
    if (scratch_acquire(c, s) != cudaSuccess) return fail(LG_ECUDA, "stream wait failed");
    rc = dock_device(c, pk->dev, bd, od, p, nmax, rmax, c->scratch, s, &c->stats, tev, nullptr, cmask, graph_ok);
    if (scratch_release(c, s) != cudaSuccess && rc == LG_OK) rc = fail(LG_ECUDA, "event record failed");
    if (rc) return rc;
    if (o->mem == LG_MEM_HOST) {
        Range fetch("fetch outputs");
        if ((rc = fetch_out(od, o, L, S, P, A, R, p->rigid_steps, s))) return rc;
    }
    if (b->mem == LG_MEM_HOST || o->mem == LG_MEM_HOST) {
        Range wait("wait for the stream");
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("docking: ") + cudaGetErrorString(e));
    } else {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("docking: ") + cudaGetErrorString(e));
    }
    return LG_OK;
}

int lg_score_poses(lg_ctx *c, int32_t pid, const lg_pose_batch *b, double *E, void *stream) {
    if (!c || !b || !E) return fail(LG_EINVAL, "null argument");
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if (b->mem != LG_MEM_HOST && b->mem != LG_MEM_DEVICE) return fail(LG_EINVAL, "bad mem");
    if (b->L == 0) return LG_OK;
    if (!b->atom_off || !b->xyz || !b->q || !b->type) return fail(LG_EINVAL, "null pose array");
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    PocketRec *pk = (pid >= 0 && pid < (int)c->pockets.size() && c->pockets[pid].live) ? &c->pockets[pid] : nullptr;
    if (!pk) return fail(LG_ENOPOCKET, "unknown pocket");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = b->L;
    const int32_t *aoff = b->atom_off;
    const float *xyz = b->xyz, *q = b->q;
    const uint8_t *t = b->type;
    double *dE = E;
    cudaError_t e = cudaSuccess;
    if (b->mem == LG_MEM_HOST) {
        if (b->atom_off[0] != 0) return fail(LG_EINVAL, "atom_off[0] must be 0");
        for (int l = 0; l < L; l++)
            if (b->atom_off[l + 1] < b->atom_off[l]) return fail(LG_EINVAL, "atom_off must be non-decreasing");
        const int64_t A = b->atom_off[L];
        Carve cv;
        const size_t o_a = cv.take(4 * (size_t)(L + 1)), o_x = cv.take(12 * (size_t)A), o_q = cv.take(4 * (size_t)A);
        const size_t o_t = cv.take((size_t)A), o_e = cv.take(8 * (size_t)L);
        if (c->in_buf.ensure(cv.off)) return fail(LG_ENOMEM, "staging allocation failed");
        char *base = (char *)c->in_buf.p;
        e = cudaMemcpyAsync(base + o_a, aoff, 4 * (size_t)(L + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && A) e = cudaMemcpyAsync(base + o_x, xyz, 12 * (size_t)A, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && A) e = cudaMemcpyAsync(base + o_q, q, 4 * (size_t)A, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && A) e = cudaMemcpyAsync(base + o_t, t, (size_t)A, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("pose upload: ") + cudaGetErrorString(e));
        aoff = (const int32_t *)(base + o_a);
        xyz = (const float *)(base + o_x);
        q = (const float *)(base + o_q);
        t = (const uint8_t *)(base + o_t);
        dE = (double *)(base + o_e);
    }
    if ((e = launch_score_poses(pk->dev, L, aoff, xyz, q, t, dE, s)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("score launch: ") + cudaGetErrorString(e));
    if (b->mem == LG_MEM_HOST) {
        e = cudaMemcpyAsync(E, dE, 8 * (size_t)L, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(LG_ECUDA, std::string("scoring: ") + cudaGetErrorString(e));
    }
    return LG_OK;
}

// Device name and SM count that a tuning text belongs to.
static std::string tune_device_name(lg_ctx *c) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return std::string();
    std::string n;
    for (const char *q = prop.name; *q; ++q)
        if (*q != '"' && *q != '\\' && (unsigned char)*q >= 32) n += *q;  // nothing to escape in the text
    return n;
}

int lg_tune_export(lg_ctx *c, char *buf, int64_t cap, int64_t *len) {
    if (!c || !len || (cap > 0 && !buf)) return fail(LG_EINVAL, "null argument");
    std::string t = "{\"device\": \"" + tune_device_name(c) + "\", \"sms\": " + std::to_string(ctx_num_sms(c)) +
                    ", \"entries\": [";
    {
        std::lock_guard<std::mutex> g(c->tune_mu);
        bool first = true;
        for (const auto &kv : c->tune) {
            t += first ? "[" : ", [";
            first = false;
            for (int v : kv.first) t += std::to_string(v) + ", ";
            t += std::to_string(kv.second.first) + ", " + std::to_string(kv.second.second) + "]";
        }
    }
    t += "]}";
    *len = (int64_t)t.size();
    if (cap < (int64_t)t.size() + 1) return fail(LG_EINVAL, "buffer too small for the tuning text");
    memcpy(buf, t.c_str(), t.size() + 1);
    return LG_OK;
}

int lg_tune_import(lg_ctx *c, const char *text) {
    if (!c || !text) return fail(LG_EINVAL, "null argument");
    const std::string t(text);
    auto field = [&](const char *name) -> size_t {  // position after "name":
        const size_t k = t.find(std::string("\"") + name + "\"");
        if (k == std::string::npos) return k;
        const size_t colon = t.find(':', k);
        return colon == std::string::npos ? colon : colon + 1;
    };
    size_t k = field("device");
    if (k == std::string::npos) return fail(LG_EINVAL, "tuning text: no device");
    const size_t q0 = t.find('"', k), q1 = q0 == std::string::npos ? q0 : t.find('"', q0 + 1);
    if (q1 == std::string::npos) return fail(LG_EINVAL, "tuning text: bad device");
    if (t.substr(q0 + 1, q1 - q0 - 1) != tune_device_name(c)) return fail(LG_EINVAL, "tuning text is for another device");
    k = field("sms");
    if (k == std::string::npos || atoi(t.c_str() + k) != ctx_num_sms(c))
        return fail(LG_EINVAL, "tuning text is for another SM count");
    k = field("entries");
    if (k == std::string::npos) return fail(LG_EINVAL, "tuning text: no entries");
    // entries: a list of lists of 10 integers (9: an entry without the
    // restart tile, 4 lanes per restart)
    std::vector<std::pair<std::array<int, 8>, std::pair<int, int>>> got;
    std::vector<long> cur;
    int depth = 0;
    for (size_t i = k; i < t.size(); ++i) {
        const char ch = t[i];
        if (ch == '[') {
            if (++depth > 2) return fail(LG_EINVAL, "tuning text: nesting");
            if (depth == 2) cur.clear();
        } else if (ch == ']') {
            if (depth == 2) {
                if (cur.size() != 9 && cur.size() != 10)
                    return fail(LG_EINVAL, "tuning text: an entry is not 10 integers");
                std::array<int, 8> key;
                for (int j = 0; j < 8; ++j) key[j] = (int)cur[j];
                const int lanes = cur.size() == 10 ? (int)cur[8] : kLanesPerRestart, w = (int)cur.back();
                if (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16)
                    return fail(LG_EINVAL, "tuning text: lanes per restart not 2, 4, 8 or 16");
                if (w < 1 || w > max_warps_of(lanes) || (w & (w - 1)) != 0)
                    return fail(LG_EINVAL, "tuning text: warps per CTA not a power of 2 within the tile's bound");
                if (key[0] < -1 || key[0] >= kSizeClasses || key[1] < 1 || key[2] < 0 || key[3] < 1 || key[4] < 1)
                    return fail(LG_EINVAL, "tuning text: bad key");
                if (lanes != kLanesPerRestart && (key[5] != 0 || key[7] >= 2))
                    return fail(LG_EINVAL, "tuning text: that restart tile exists for single-pocket launches without ranking only");
                got.push_back({key, {lanes, w}});
            }
            if (--depth == 0) break;
        } else if (ch == '-' || (ch >= '0' && ch <= '9')) {
            if (depth != 2) return fail(LG_EINVAL, "tuning text: number outside an entry");
            char *end = nullptr;
            cur.push_back(strtol(t.c_str() + i, &end, 10));
            i = (size_t)(end - t.c_str()) - 1;
        } else if (ch != ',' && ch != ' ' && ch != '\n' && ch != '\t' && ch != '\r') {
            return fail(LG_EINVAL, "tuning text: unexpected character");
        }
    }
    if (depth != 0) return fail(LG_EINVAL, "tuning text: unterminated entries");
    std::lock_guard<std::mutex> g(c->tune_mu);
    for (const auto &e : got) c->tune[e.first] = e.second;
    return LG_OK;
}

int lg_get_stats(lg_ctx *c, lg_stats *out) {
    if (!c || !out) return fail(LG_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    harvest_timing(c);
    *out = c->stats;
    serve_stats(c, out);
    return LG_OK;
}

int lg_set_option(lg_ctx *c, const char *key, int64_t v) {
    if (!c || !key) return fail(LG_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(c->mu);
    if (!strcmp(key, "timing")) {
        cudaSetDevice(c->device);
        harvest_timing(c);
        c->timing = v != 0;
        c->stats.dock_calls = 0;
        c->stats.dock_ms_total = 0.0;
    } else if (!strcmp(key, "warps_per_cta")) {
        if (v < 0 || v > 32) return fail(LG_EINVAL, "warps_per_cta must be in [0, 32]");
        c->warps_opt = (int)v;
    } else if (!strcmp(key, "restart_lanes")) {
        if (v != 0 && v != 2 && v != 4 && v != 8 && v != 16)
            return fail(LG_EINVAL, "restart_lanes must be 0, 2, 4, 8 or 16");
        c->lanes_opt = (int)v;
    } else if (!strcmp(key, "serve_max_merge")) {
        if (v < 1 || v > (1 << 20)) return fail(LG_EINVAL, "serve_max_merge must be in [1, 2^20]");
        c->serve_max_merge = (int)v;
    } else if (!strcmp(key, "serve_cross_pocket")) {
        c->serve_cross_pocket = v != 0;
    } else if (!strcmp(key, "serve_device_loop")) {
        if (c->serve_device_loop != (v != 0)) {
            c->serve_device_loop = v != 0;
            serve_stop(c);  // the next submission starts a worker of the other kind
        }
    } else if (!strcmp(key, "serve_loop_lanes")) {
        if (v != 0 && v != 4 && v != 16) return fail(LG_EINVAL, "serve_loop_lanes must be 0, 4 or 16");
        if (c->serve_loop_lanes != (int)v) {
            c->serve_loop_lanes = (int)v;
            serve_stop(c);  // the next submission starts a loop with the new tile
        }
    } else if (!strcmp(key, "serve_loop_idle_ms")) {
        if (v < 1 || v > 60000) return fail(LG_EINVAL, "serve_loop_idle_ms must be in [1, 60000]");
        c->serve_loop_idle_ms = (int)v;
    } else if (!strcmp(key, "serve_max_inflight")) {
        if (v < 1 || v > 64) return fail(LG_EINVAL, "serve_max_inflight must be in [1, 64]");
        c->serve_max_inflight = (int)v;
    } else if (!strcmp(key, "graphs")) {
        cudaSetDevice(c->device);
        if (v < 0 || v > 2) return fail(LG_EINVAL, "graphs must be 0, 1 or 2");
        c->graphs = (int)v;
        for (auto &g : c->graph_cache) cudaGraphExecDestroy(g.exec);
        c->graph_cache.clear();
        c->graph_seen.clear();
    } else if (!strcmp(key, "size_classes")) {
        c->size_classes = v != 0;
    } else if (!strcmp(key, "autotune")) {
        c->autotune = v != 0;
        std::lock_guard<std::mutex> tg(c->tune_mu);
        c->tune.clear();
    } else if (!strcmp(key, "multi_order")) {
        if (v != 0 && v != 1) return fail(LG_EINVAL, "multi_order must be 0 or 1");
        c->multi_pocket_major = v == 0 ? 1 : 0;
    } else if (!strcmp(key, "l2_window")) {
        c->l2_window = v != 0;
        cudaSetDevice(c->device);
        for (auto &g : c->graph_cache) cudaGraphExecDestroy(g.exec);  // captured launches carry the old choice
        c->graph_cache.clear();
    } else if (!strcmp(key, "pocket_pack_host")) {
        c->pack_host = v != 0;
    } else if (!strcmp(key, "serve_mem_reserve_mb")) {
        if (v < 0) return fail(LG_EINVAL, "serve_mem_reserve_mb must be >= 0");
        c->serve_reserve_mb = v;
    } else {
        return fail(LG_EINVAL, std::string("unknown option ") + key);
    }
    return LG_OK;
}

int lg_diag_fp32_peak(lg_ctx *c, int32_t reps, double *tflops, double *seconds) {
    if (!c || !tflops || reps < 1 || reps > 100) return fail(LG_EINVAL, "bad argument");
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    const int blocks = ctx_num_sms(c) * 8, iters = 1 << 18;
    float *out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * 256 * (size_t)blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    double best = 0.0, total = 0.0;
    if (e == cudaSuccess) e = launch_fp32_peak(out, blocks, iters, 0);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(t0, 0);
        e = launch_fp32_peak(out, blocks, iters, 0);
        cudaEventRecord(t1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && ms > 0.0f) {
            const double flop = 2.0 * 8.0 * iters * 256.0 * blocks;
            best = std::max(best, flop / (ms * 1e-3) / 1e12);
            total += ms * 1e-3;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("FP32 peak: ") + cudaGetErrorString(e));
    *tflops = best;
    if (seconds) *seconds = total;
    return LG_OK;
}

int lg_diag_pocket_cells(lg_ctx *c, int32_t pid, float *cell_o, float *cell_ve) {
    if (!c || !cell_o || !cell_ve) return fail(LG_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(c->mu);
    if (pid < 0 || pid >= (int)c->pockets.size() || !c->pockets[pid].live) return fail(LG_EINVAL, "unknown pocket");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    const PocketDev &pd = c->pockets[pid].dev;
    const size_t n3 = (size_t)pd.n * pd.n * pd.n;
    cudaError_t e = cudaMemcpy(cell_o, pd.cell_o, 32 * n3, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(cell_ve, pd.cell_ve, 64 * n3, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("pocket cells: ") + cudaGetErrorString(e));
    return LG_OK;
}

int lg_diag_philox(lg_ctx *c, int32_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int32_t use_curand) {
    if (!c || n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(LG_EINVAL, "bad argument");
    if (n == 0) return LG_OK;
    std::lock_guard<std::mutex> g(c->mu);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(LG_ECUDA, "cudaSetDevice failed");
    cudaError_t e = launch_diag_philox(n, ctr, key, out, use_curand, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("philox: ") + cudaGetErrorString(e));
    return LG_OK;
}

}  // extern "C"
