// Serving loop of liblgdock: lg_stream_submit / lg_stream_poll / lg_stream_wait.
//
// The paper streams a chemical library through a fixed binding site with an
// asynchronous reader -> docker -> writer pipeline whose stages talk through
// thread-safe queues (Sec. 3.2).  Here one worker thread per context takes
// requests from a host queue, merges the queued requests that share a pocket
// and parameters into one batch (with the option serve_cross_pocket, requests
// aimed at different pockets too: each ligand is then docked against its own
// request's pocket in the same launch), and keeps up to `serve_max_inflight` such
// batches on the device at once, each on its own stream (continuous batching:
// a request that arrives while others run is admitted as soon as a slot and
// enough free device memory are there).  Results are per ligand, so a
// ligand's result does not depend on which requests it was merged with.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstddef>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>

#include "lg_ring.h"
#include "lg_runtime.h"

namespace lg {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    PocketDev pocket{};
    lg_dock_params params{};
    lg_dock_result out{};
    int L = 0;
    int64_t A = 0, R = 0;
    int nmax = 0, rmax = 0;
    std::vector<int32_t> atom_off, rot_off;
    std::vector<float> x, y, z, q;
    std::vector<uint8_t> type;
    std::vector<int16_t> parent, rot_child;
    std::vector<uint64_t> uid;
    int state = LG_REQ_QUEUED;
    double t_submit = 0.0, t_done = 0.0;
};

struct PinnedBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n) {
        if (n <= cap) return 0;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, n) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        cap = n;
        return 0;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

struct Slot {
    bool busy = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf in, out, scratch, lp;  // lp: pocket slot of every merged ligand
    PinnedBuf hin, hout, hlp;
    std::vector<std::shared_ptr<Request>> reqs;
    int L = 0;
    int64_t A = 0, R = 0;
    lg_dock_result hres{};  // merged host result (views into hout)
};

struct DeviceLoop;  // the device-resident loop's state (below)

struct Server {
    lg_ctx *ctx = nullptr;
    DeviceLoop *loop = nullptr;  // set when the device-resident loop serves the requests
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable done_cv;  // wakes waiters
    bool stop = false;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    static constexpr size_t kMaxQueued = 1 << 16;
};

// Requests that can share one launch: same parameters and the same optional
// outputs, and the same pocket unless cross-pocket merging is on (each ligand
// is then docked against its own request's pocket).
static bool same_kind(const Request &a, const Request &b, bool cross_pocket) {
    return (cross_pocket || a.pocket.cell_o == b.pocket.cell_o) && a.params.restarts == b.params.restarts &&
           a.params.passes == b.params.passes && a.params.seed == b.params.seed &&
           a.params.d_clash == b.params.d_clash && a.params.max_atoms == b.params.max_atoms &&
           a.params.max_rot == b.params.max_rot && (a.out.pose != nullptr) == (b.out.pose != nullptr) &&
           (a.out.tors_idx != nullptr) == (b.out.tors_idx != nullptr) &&
           (a.out.restart_score != nullptr) == (b.out.restart_score != nullptr) &&
           (a.out.restart_tors != nullptr) == (b.out.restart_tors != nullptr) &&
           a.params.cluster_rmsd == b.params.cluster_rmsd && a.params.rescore_top == b.params.rescore_top &&
           (a.out.rank != nullptr) == (b.out.rank != nullptr) &&
           (a.out.leader != nullptr) == (b.out.leader != nullptr) &&
           (a.out.restart_geo != nullptr) == (b.out.restart_geo != nullptr) &&
           a.params.rigid_steps == b.params.rigid_steps && a.params.rigid_shift == b.params.rigid_shift &&
           (a.out.restart_rigid != nullptr) == (b.out.restart_rigid != nullptr);
}

// Pinned CSR image of the requests' ligands, concatenated in order (offsets
// rebased); mb views it.
static int build_input_image(PinnedBuf &hin, const std::vector<std::shared_ptr<Request>> &reqs, int L, int64_t A,
                             int64_t R, lg_ligand_batch *mb) {
    const size_t bytes_in = 8 * (size_t)(L + 1) + 8 * (size_t)L + 19 * (size_t)A + 2 * (size_t)R + 64;
    if (hin.ensure(bytes_in)) return fail(LG_ENOMEM, "pinned staging allocation failed");
    char *h = (char *)hin.p;
    int32_t *aoff = (int32_t *)h;
    int32_t *roff = aoff + (L + 1);
    uint64_t *uid = (uint64_t *)(((uintptr_t)(roff + L + 1) + 7) & ~(uintptr_t)7);
    float *x = (float *)(uid + L), *y = x + A, *z = y + A, *q = z + A;
    int16_t *par = (int16_t *)(q + A);
    int16_t *rc = par + A;
    uint8_t *ty = (uint8_t *)(rc + R);
    int l0 = 0;
    int64_t a0 = 0, k0 = 0;
    aoff[0] = 0;
    roff[0] = 0;
    for (auto &r : reqs) {
        for (int l = 0; l < r->L; l++) {
            aoff[l0 + l + 1] = (int32_t)(a0 + r->atom_off[l + 1]);
            roff[l0 + l + 1] = (int32_t)(k0 + r->rot_off[l + 1]);
        }
        memcpy(uid + l0, r->uid.data(), 8 * (size_t)r->L);
        memcpy(x + a0, r->x.data(), 4 * (size_t)r->A);
        memcpy(y + a0, r->y.data(), 4 * (size_t)r->A);
        memcpy(z + a0, r->z.data(), 4 * (size_t)r->A);
        memcpy(q + a0, r->q.data(), 4 * (size_t)r->A);
        memcpy(par + a0, r->parent.data(), 2 * (size_t)r->A);
        memcpy(ty + a0, r->type.data(), (size_t)r->A);
        if (r->R) memcpy(rc + k0, r->rot_child.data(), 2 * (size_t)r->R);
        l0 += r->L;
        a0 += r->A;
        k0 += r->R;
    }
    memset(mb, 0, sizeof(*mb));
    mb->L = L;
    mb->mem = LG_MEM_HOST;
    mb->atom_off = aoff;
    mb->rot_off = roff;
    mb->uid = uid;
    mb->x = x; mb->y = y; mb->z = z; mb->q = q;
    mb->type = ty;
    mb->parent = par;
    mb->rot_child = rc;
    return LG_OK;
}

// Pinned output image of L ligands (A atoms, R torsional bonds) holding the
// outputs that requests of r0's kind ask for; hr views it.
static int build_output_image(PinnedBuf &hout, const Request &r0, int L, int64_t A, int64_t R, lg_dock_result *hr) {
    const int S = r0.params.restarts, P = r0.params.passes, Rs = r0.params.rigid_steps;
    memset(hr, 0, sizeof(*hr));
    hr->mem = LG_MEM_HOST;
    size_t ob = 8 * (size_t)L + 4 * (size_t)L + 4 * (size_t)L;
    const bool want_t = r0.out.tors_idx, want_p = r0.out.pose, want_rs = r0.out.restart_score,
               want_rt = r0.out.restart_tors, want_rk = r0.out.rank, want_ld = r0.out.leader,
               want_g = r0.out.restart_geo, want_rg = r0.out.restart_rigid;
    ob += want_rk ? 4 * (size_t)L * S : 0;
    ob += want_ld ? 4 * (size_t)L * S : 0;
    ob += want_g ? 8 * (size_t)L * S : 0;
    ob += want_t ? (size_t)P * R : 0;
    ob += want_rg ? (size_t)L * S * P * Rs : 0;
    ob += want_p ? 12 * (size_t)A : 0;
    ob += want_rs ? 8 * (size_t)L * S : 0;
    ob += want_rt ? (size_t)S * P * R : 0;
    if (hout.ensure(ob + 64)) return fail(LG_ENOMEM, "pinned result allocation failed");
    char *o = (char *)hout.p;
    hr->score = (double *)o; o += 8 * (size_t)L;
    if (want_rs) { hr->restart_score = (double *)o; o += 8 * (size_t)L * S; }
    if (want_g) { hr->restart_geo = (double *)o; o += 8 * (size_t)L * S; }
    hr->best_restart = (int32_t *)o; o += 4 * (size_t)L;
    hr->status = (int32_t *)o; o += 4 * (size_t)L;
    if (want_rk) { hr->rank = (int32_t *)o; o += 4 * (size_t)L * S; }
    if (want_ld) { hr->leader = (int32_t *)o; o += 4 * (size_t)L * S; }
    if (want_p) { hr->pose = (float *)o; o += 12 * (size_t)A; }
    if (want_t) { hr->tors_idx = (uint8_t *)o; o += (size_t)P * R; }
    if (want_rt) { hr->restart_tors = (uint8_t *)o; o += (size_t)S * P * R; }
    if (want_rg) { hr->restart_rigid = (uint8_t *)o; }
    return LG_OK;
}

// Concatenate the requests into the slot's pinned buffer and launch them.
static int launch_slot(Server *sv, Slot &sl) {
    Range range("serve: merged launch");
    lg_ctx *c = sv->ctx;
    const Request &r0 = *sl.reqs[0];
    const int S = r0.params.restarts, P = r0.params.passes, Rs = r0.params.rigid_steps;
    int L = 0, nmax = 1, rmax = 1;
    int64_t A = 0, R = 0;
    for (auto &r : sl.reqs) {
        L += r->L;
        A += r->A;
        R += r->R;
        nmax = std::max(nmax, r->nmax);
        rmax = std::max(rmax, r->rmax);
    }
    sl.L = L;
    sl.A = A;
    sl.R = R;
    lg_ligand_batch mb;
    int rc2;
    if ((rc2 = build_input_image(sl.hin, sl.reqs, L, A, R, &mb))) return rc2;
    lg_dock_result &hr = sl.hres;
    if ((rc2 = build_output_image(sl.hout, r0, L, A, R, &hr))) return rc2;

    cudaSetDevice(c->device);
    BatchDev bd;
    OutDev od;
    if ((rc2 = stage_batch(sl.in, &mb, A, R, &bd, sl.stream))) return rc2;
    if ((rc2 = stage_out(sl.out, &hr, L, S, P, A, R, Rs, &od))) return rc2;
    lg_dock_params p = r0.params;
    p.mode = LG_MODE_BATCHED;
    lg_stats st{};
    // distinct pockets of the merged requests (the merge keeps them <= LG_MAX_MULTI_POCKETS)
    std::vector<PocketDev> pks;
    std::vector<int> slot_of;
    for (auto &r : sl.reqs) {
        int k = 0;
        while (k < (int)pks.size() && pks[k].cell_o != r->pocket.cell_o) k++;
        if (k == (int)pks.size()) pks.push_back(r->pocket);
        slot_of.push_back(k);
    }
    if (pks.size() == 1) {
        if ((rc2 = dock_device(c, r0.pocket, bd, od, &p, nmax, rmax, sl.scratch, sl.stream, &st, nullptr))) return rc2;
    } else {
        if (sl.hlp.ensure(4 * (size_t)L) || sl.lp.ensure(4 * (size_t)L))
            return fail(LG_ENOMEM, "pocket index allocation failed");
        int32_t *hl = (int32_t *)sl.hlp.p;
        int l0 = 0;
        for (size_t q = 0; q < sl.reqs.size(); q++) {
            for (int l = 0; l < sl.reqs[q]->L; l++) hl[l0 + l] = slot_of[q];
            l0 += sl.reqs[q]->L;
        }
        if (cudaMemcpyAsync(sl.lp.p, hl, 4 * (size_t)L, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return fail(LG_ECUDA, "pocket index upload failed");
        std::unique_ptr<MultiDev> m(new MultiDev());
        memset(m.get(), 0, sizeof(MultiDev));
        m->np = (int)pks.size();
        for (int k = 0; k < m->np; k++) m->pk[k] = pks[k];
        m->lig_pocket = (const int32_t *)sl.lp.p;
        if ((rc2 = dock_device(c, pks[0], bd, od, &p, nmax, rmax, sl.scratch, sl.stream, &st, nullptr, m.get())))
            return rc2;
    }
    if ((rc2 = fetch_out(od, &hr, L, S, P, A, R, Rs, sl.stream))) return rc2;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return fail(LG_ECUDA, "event record failed");
    return LG_OK;
}

// Copy merged results (hr, the requests in order) into each request's own
// output buffers and mark the requests done (or failed).
static void scatter_outputs(const lg_dock_result &hr, std::vector<std::shared_ptr<Request>> &reqs, bool ok) {
    int l0 = 0;
    int64_t a0 = 0, k0 = 0;
    const double t = now_s();
    for (auto &r : reqs) {
        const int S = r->params.restarts, P = r->params.passes;
        if (ok) {
            memcpy(r->out.score, hr.score + l0, 8 * (size_t)r->L);
            memcpy(r->out.best_restart, hr.best_restart + l0, 4 * (size_t)r->L);
            memcpy(r->out.status, hr.status + l0, 4 * (size_t)r->L);
            if (r->out.tors_idx && r->R) memcpy(r->out.tors_idx, hr.tors_idx + (size_t)P * k0, (size_t)P * r->R);
            if (r->out.pose) memcpy(r->out.pose, hr.pose + 3 * a0, 12 * (size_t)r->A);
            if (r->out.restart_score)
                memcpy(r->out.restart_score, hr.restart_score + (size_t)S * l0, 8 * (size_t)S * r->L);
            if (r->out.restart_tors && r->R)
                memcpy(r->out.restart_tors, hr.restart_tors + (size_t)S * P * k0, (size_t)S * P * r->R);
            if (r->out.rank) memcpy(r->out.rank, hr.rank + (size_t)S * l0, 4 * (size_t)S * r->L);
            if (r->out.leader) memcpy(r->out.leader, hr.leader + (size_t)S * l0, 4 * (size_t)S * r->L);
            if (r->out.restart_geo)
                memcpy(r->out.restart_geo, hr.restart_geo + (size_t)S * l0, 8 * (size_t)S * r->L);
            if (r->out.restart_rigid) {
                const size_t per = (size_t)S * P * r->params.rigid_steps;
                memcpy(r->out.restart_rigid, hr.restart_rigid + per * l0, per * r->L);
            }
        }
        l0 += r->L;
        a0 += r->A;
        k0 += r->R;
        r->t_done = t;
        r->state = ok ? LG_REQ_DONE : LG_REQ_FAILED;
        // the request's copy of the batch is no longer needed
        std::vector<float>().swap(r->x);
        std::vector<float>().swap(r->y);
        std::vector<float>().swap(r->z);
        std::vector<float>().swap(r->q);
        std::vector<int16_t>().swap(r->parent);
        std::vector<int16_t>().swap(r->rot_child);
        std::vector<uint8_t>().swap(r->type);
    }
}

// Split the merged results back into each request's output buffers.
static void finish_slot(Slot &sl, bool ok) {
    scatter_outputs(sl.hres, sl.reqs, ok);
    sl.reqs.clear();
    sl.busy = false;
}

static size_t request_device_bytes(const Request &r) {
    const size_t S = r.params.restarts, P = r.params.passes;
    return 40 * (size_t)r.L + 19 * (size_t)r.A + 2 * (size_t)r.R + (r.out.pose ? 12 * (size_t)r.A : 0) +
           (r.out.tors_idx ? P * r.R : 0) + (r.out.restart_score ? 8 * S * r.L : 0) +
           (r.out.restart_tors ? S * P * r.R : 0) + (r.out.rank ? 4 * S * r.L : 0) +
           (r.out.leader ? 4 * S * r.L : 0) + (r.out.restart_geo ? 8 * S * r.L : 0) +
           (r.out.restart_rigid ? S * P * r.params.rigid_steps * r.L : 0) + 8 * (size_t)r.L + 4096;
}

// Device scratch of a merged batch (dock_device's buffer): cost order,
// centroids, subtree ends and, with pose ranking, one pose slot per CTA of
// the widest launch the call may make (at most 32 CTAs per SM, and never
// more slots than ligands).
static size_t merged_scratch_bytes(lg_ctx *c, const Request &r, int L, int nmax, int rmax) {
    const bool ranking = ranking_on(&r.params);
    const int slots = ranking ? std::max(1, std::min(L, 32 * ctx_num_sms(c))) : 0;
    return scratch_bytes(L, rmax, slots, r.params.restarts, r.params.passes, nmax);
}

static void worker(Server *sv) {
    lg_ctx *c = sv->ctx;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progressed = false;
        // completions
        for (auto &sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish_slot(sl, q == cudaSuccess);
            if (q != cudaSuccess) cudaGetLastError();
            progressed = true;
        }
        if (progressed) sv->done_cv.notify_all();
        // admissions
        int busy = 0;
        for (auto &sl : sv->slots) busy += sl.busy;
        while (!sv->queue.empty()) {
            Slot *free_sl = nullptr;
            for (auto &sl : sv->slots)
                if (!sl.busy) {
                    free_sl = &sl;
                    break;
                }
            if (!free_sl) break;
            // One merged batch per kind of request: the first queued request of
            // a kind not yet tried in this round seeds it, and the later queued
            // requests of the same kind join it in arrival order.  A batch that
            // does not fit in free device memory stays queued where it is (no
            // request moves) and the next kind is tried, so a large request
            // waiting for memory does not hold back smaller ones of other kinds.
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            const size_t reserve = (size_t)c->serve_reserve_mb << 20;
            const size_t have = free_sl->in.cap + free_sl->out.cap + free_sl->scratch.cap;
            const int max_merge = c->serve_max_merge;
            std::vector<const Request *> tried;
            std::vector<size_t> take_idx;
            for (size_t seed = 0; seed < sv->queue.size() && take_idx.empty(); ++seed) {
                const Request &rs = *sv->queue[seed];
                bool seen = false;
                for (const Request *t : tried) seen = seen || same_kind(*t, rs, c->serve_cross_pocket);
                if (seen) continue;
                tried.push_back(&rs);
                std::vector<size_t> idx;
                std::vector<const float4 *> pockets;  // distinct pockets of the merged batch
                int Lm = 0, nm = 1, rm = 1;
                size_t bytes = 0;
                for (size_t i = seed; i < sv->queue.size(); ++i) {
                    const Request &r = *sv->queue[i];
                    const bool known = std::find(pockets.begin(), pockets.end(), r.pocket.cell_o) != pockets.end();
                    if (!idx.empty() && (!same_kind(rs, r, c->serve_cross_pocket) || Lm + r.L > max_merge ||
                                         (!known && (int)pockets.size() >= LG_MAX_MULTI_POCKETS)))
                        continue;
                    if (!known) pockets.push_back(r.pocket.cell_o);
                    idx.push_back(i);
                    Lm += r.L;
                    nm = std::max(nm, r.nmax);
                    rm = std::max(rm, r.rmax);
                    bytes += request_device_bytes(r);
                    if (Lm >= max_merge) break;
                }
                bytes += merged_scratch_bytes(c, rs, Lm, nm, rm);
                // admission by free device memory (an idle device always admits)
                const size_t need = bytes > have ? bytes - have : 0;
                if (busy > 0 && need > 0 && need + reserve > fr) continue;
                take_idx = idx;
            }
            if (take_idx.empty()) break;  // nothing fits until a batch in flight finishes
            std::vector<std::shared_ptr<Request>> take;
            for (size_t i : take_idx) take.push_back(sv->queue[i]);
            for (size_t j = take_idx.size(); j-- > 0;) sv->queue.erase(sv->queue.begin() + take_idx[j]);
            // requests for the same pocket side by side: the merged batch is
            // docked in this order, one pocket's grids in L2 at a time
            std::stable_sort(take.begin(), take.end(),
                             [](const std::shared_ptr<Request> &x, const std::shared_ptr<Request> &y) {
                                 return (uintptr_t)x->pocket.cell_o < (uintptr_t)y->pocket.cell_o;
                             });
            for (auto &r : take) r->state = LG_REQ_RUNNING;
            free_sl->reqs = take;
            free_sl->busy = true;
            lk.unlock();
            const int rc = launch_slot(sv, *free_sl);
            lk.lock();
            if (rc != LG_OK) {
                cudaStreamSynchronize(free_sl->stream);
                finish_slot(*free_sl, false);
                sv->done_cv.notify_all();
            } else {
                busy++;
            }
        }
        if (sv->stop && sv->queue.empty() && busy == 0) break;
        if (busy > 0)
            sv->cv.wait_for(lk, std::chrono::microseconds(100));
        else if (sv->queue.empty() && !sv->stop)
            sv->cv.wait(lk);
    }
}

// ======================================================================= device-resident loop
// With the option serve_device_loop (the default) requests are not merged into
// launches: one persistent launch of k_serve_loop stays on the device and
// docks ligands as they are admitted.  Admitting a request copies its ligands
// into a ring arena of CSR arrays in device memory and reserves the same
// ranges of an output arena in mapped pinned host memory; then its descriptor
// (arena slot, pocket) and the raised published-ligand count follow, all by
// copies on the feed stream, in that order.  The kernel writes each ligand's
// outputs straight into the output arena and raises the request's completion
// flag in mapped host memory, which the worker polls; it then copies the
// request's outputs to the caller's buffers.  Arena ranges are released in
// admission order.  The launch's arguments hold the arenas and a table of
// pockets, so a request for a pocket not yet in the table relaunches the loop
// with the table extended.  CTAs that find no ligand for serve_loop_idle_ms
// leave, so an idle loop ends by itself; the worker relaunches it when work
// is pending.
constexpr int kRing = 256;  // requests in flight at most

struct RingSlot {
    bool busy = false;
    uint64_t seq = 0;
    std::vector<std::shared_ptr<Request>> reqs;  // the request (one)
    size_t slot = 0, atom = 0, tor = 0;          // its arena ranges
    PinnedBuf hin;                               // its pinned staging (from the pool)
};

struct DeviceLoop {
    bool ready = false;       // streams, control block and host buffers exist
    bool configured = false;  // a kind is set up (layouts, scratch, arenas)
    bool running = false;     // a launch may still be on the device
    std::shared_ptr<Request> kind;  // a request of the kind the loop serves
    int nmax = 0, rmax = 0, W = 1, occ = 0, smem = 0, grid = 0;
    // the kind's restart tiles: [0] 4 lanes per restart (throughput), [1] 16
    // lanes (latency; not for pose ranking); `cur` is the one launched
    struct Tile {
        int lanes = 0, W = 0, occ = 0, smem = 0, grid = 0;
        Layout ly;
        LayoutRT lrt;
    } tiles[2];
    int ntiles = 1, cur = 0, held_n = 0;
    bool held_dirty = false;  // a launch of this kind ran: the held array may hold claimed ligands
    int stale = 0;            // launches in a row that ended idle without a request finishing
    bool adaptive = false;    // switch tiles by the backlog
    double low_since = -1.0;  // since when the backlog has been low (throughput tile)
    int64_t switches = 0;
    DockArgs args;
    std::vector<PocketDev> table;  // pockets of the launch's table
    bool table_launched = false;   // the running launch has the whole table
    DevBuf scratch, ctl, held, arena;
    void *host = nullptr;     // mapped pinned memory: flags, copy sources, exit status
    void *out = nullptr;      // mapped pinned output arena
    size_t cap_l = 0, cap_a = 0, cap_r = 0;  // arena capacities: ligand slots, atoms, torsional bonds
    RingAlloc ra_l, ra_a, ra_r;
    lg_dock_result out_h{};   // host views of the output arena
    cudaStream_t stream = nullptr, feed = nullptr;
    cudaEvent_t ended = nullptr, fed = nullptr;
    std::vector<RingSlot> ring;
    std::multimap<size_t, void *> spare;  // pinned staging buffers not in use, by capacity (freed at release)
    size_t mem_free = 0;      // free device memory at the last query
    double mem_t = -1.0;      // time of that query
    uint64_t next_seq = 0, head = 0, tail = 0;
    int last_status = -1;
    int64_t launches = 0, items = 0;
    // the figures lg_get_stats reads while the worker runs
    std::atomic<int> a_status{-1};
    std::atomic<int64_t> a_launches{0}, a_items{0}, a_switches{0};
    // views of ctl (device) and host
    LoopCtl *d_ctl = nullptr;
    LoopDesc *d_desc = nullptr;
    uint32_t *d_done = nullptr;
    uint64_t *h_flags = nullptr, *d_flags = nullptr;
    LoopDesc *h_desc = nullptr;
    uint64_t *h_seq = nullptr, *h_tail = nullptr, *h_head = nullptr, *h_busy = nullptr;
    uint32_t *h_stop = nullptr;  // {0, 1}
    int32_t *h_status = nullptr;
};

static size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// Requests the loop's kind serves: the same parameters and optional outputs
// (any pocket) within the layout's maxima and the arenas' capacities.
static bool loop_fits(const DeviceLoop &dl, const Request &r) {
    return dl.configured && same_kind(*dl.kind, r, true) && r.nmax <= dl.nmax && r.rmax <= dl.rmax &&
           (size_t)r.L + 1 <= dl.cap_l && (size_t)r.A <= dl.cap_a && (size_t)r.R <= dl.cap_r;
}

// Pinned staging buffers come from a pool that only grows (freeing pinned
// memory can wait for the device, and allocating it is slow): the smallest
// spare buffer that fits, else a new one of at least 64 KiB, rounded up to a
// power of two.
static int pinned_get(DeviceLoop &dl, PinnedBuf &b, size_t n) {
    auto it = dl.spare.lower_bound(n);
    if (it != dl.spare.end()) {
        b.cap = it->first;
        b.p = it->second;
        dl.spare.erase(it);
        return 0;
    }
    size_t cap = 64 << 10;
    while (cap < n) cap <<= 1;
    if (cudaMallocHost(&b.p, cap) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        b.cap = 0;
        return -1;
    }
    b.cap = cap;
    return 0;
}

static void pinned_put(DeviceLoop &dl, PinnedBuf &b) {
    if (b.p) dl.spare.emplace(b.cap, b.p);
    b.p = nullptr;
    b.cap = 0;
}

static int loop_setup(lg_ctx *c, DeviceLoop &dl) {
    if (dl.ready) return LG_OK;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&dl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&dl.feed, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&dl.ended, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&dl.fed, cudaEventDisableTiming)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("serving loop streams: ") + cudaGetErrorString(e));
    const size_t ctl_bytes = al256(sizeof(LoopCtl)) + al256(kRing * sizeof(LoopDesc)) + al256(4 * kRing);
    if (dl.ctl.ensure(ctl_bytes)) return fail(LG_ENOMEM, "serving loop control block allocation failed");
    char *d = (char *)dl.ctl.p;
    dl.d_ctl = (LoopCtl *)d;
    dl.d_desc = (LoopDesc *)(d + al256(sizeof(LoopCtl)));
    dl.d_done = (uint32_t *)(d + al256(sizeof(LoopCtl)) + al256(kRing * sizeof(LoopDesc)));
    const size_t host_bytes = al256(8 * kRing) + al256(kRing * sizeof(LoopDesc)) + 3 * al256(8 * kRing) + 256;
    if (cudaHostAlloc(&dl.host, host_bytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return fail(LG_ENOMEM, "serving loop host buffers allocation failed");
    }
    memset(dl.host, 0, host_bytes);
    char *h = (char *)dl.host;
    dl.h_flags = (uint64_t *)h;
    h += al256(8 * kRing);
    dl.h_desc = (LoopDesc *)h;
    h += al256(kRing * sizeof(LoopDesc));
    dl.h_seq = (uint64_t *)h;
    h += al256(8 * kRing);
    dl.h_tail = (uint64_t *)h;
    h += al256(8 * kRing);
    dl.h_head = (uint64_t *)h;
    h += al256(8 * kRing);
    dl.h_busy = (uint64_t *)h;
    dl.h_stop = (uint32_t *)(h + 8);
    dl.h_status = (int32_t *)(h + 16);
    *dl.h_busy = kDescBusy;
    dl.h_stop[0] = 0u;
    dl.h_stop[1] = 1u;
    void *dflags = nullptr;
    if ((e = cudaHostGetDevicePointer(&dflags, dl.h_flags, 0)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("serving loop flags: ") + cudaGetErrorString(e));
    dl.d_flags = (uint64_t *)dflags;
    dl.ring.resize(kRing);
    (void)c;
    dl.ready = true;
    return LG_OK;
}

// Output arena of a kind (host views in dl.out_h): the outputs its requests
// ask for, laid out by arena slot, atom and torsional bond.
static size_t out_arena_bytes(const Request &r, size_t CL, size_t CA, size_t CR) {
    const size_t S = r.params.restarts, P = r.params.passes, Rs = r.params.rigid_steps;
    return al256(8 * CL) + 2 * al256(4 * CL) + (r.out.tors_idx ? al256(P * CR) : 0) +
           (r.out.pose ? al256(12 * CA) : 0) + (r.out.restart_score ? al256(8 * S * CL) : 0) +
           (r.out.restart_tors ? al256(S * P * CR) : 0) + (r.out.rank ? al256(4 * S * CL) : 0) +
           (r.out.leader ? al256(4 * S * CL) : 0) + (r.out.restart_geo ? al256(8 * S * CL) : 0) +
           (r.out.restart_rigid ? al256(S * P * Rs * CL) : 0);
}

static void loop_free_arenas(DeviceLoop &dl) {
    dl.arena.release();
    if (dl.out) cudaFreeHost(dl.out);
    dl.out = nullptr;
    dl.cap_l = dl.cap_a = dl.cap_r = 0;
}

// Make tile t the one the next launch uses (no launch on the device).
static void loop_apply_tile(DeviceLoop &dl, int t) {
    const DeviceLoop::Tile &T = dl.tiles[t];
    dl.cur = t;
    dl.args.ly = T.ly;
    dl.args.lrt = T.lrt;
    dl.args.lanes = T.lanes;
    dl.W = T.W;
    dl.occ = T.occ;
    dl.smem = T.smem;
    dl.grid = T.grid;
}

// The tile the backlog (ligands of the requests on the device) asks for.
// Claims are first come, first served, so a ligand waits for the backlog
// ahead of it. One wave of the latency tile (one ligand per SM, about half
// the throughput tile's time per ligand) clears in half the time of a
// throughput wave, and a backlog of w latency waves takes w/2 throughput
// waves; a switch costs the running CTAs' current ligands and leaves the
// loop at the other tile for the requests that follow. Hence the
// throughput tile only for a backlog above eight latency waves, and the
// latency tile again once the backlog has stayed within one wave for 5 ms.
static int loop_tile_wanted(DeviceLoop &dl, int64_t backlog, double t) {
    if (!dl.adaptive) return dl.cur;
    const int64_t wave = dl.tiles[1].grid;
    if (dl.cur == 1) {
        dl.low_since = -1.0;
        return backlog > 8 * wave ? 0 : 1;
    }
    if (backlog > wave) {
        dl.low_since = -1.0;
        return 0;
    }
    if (dl.low_since < 0.0) dl.low_since = t;
    return t - dl.low_since >= 0.005 ? 1 : 0;
}

// Set the loop up for requests of r's kind (no launch on the device, no
// request in flight): layouts for the kind's maxima, per-CTA scratch, arenas
// with room for at least r (admission by free device memory: the arena's
// size backs off until it fits next to the reserve), an empty ring and table.
static int loop_configure(lg_ctx *c, DeviceLoop &dl, const std::shared_ptr<Request> &r) {
    const lg_dock_params &p = r->params;
    dl.configured = false;
    dl.nmax = r->nmax <= class_bound(1) ? class_bound(1) : LG_MAX_ATOMS;
    dl.rmax = r->rmax <= 16 ? 16 : LG_MAX_ROT;
    DockArgs &a = dl.args;
    memset(&a, 0, sizeof(a));
    a.S = p.restarts;
    a.P = p.passes;
    a.seed_lo = (uint32_t)p.seed;
    a.seed_hi = (uint32_t)(p.seed >> 32);
    a.nmax_lim = dl.nmax;
    a.rmax_lim = dl.rmax;
    a.rigid_steps = p.rigid_steps;
    a.ranking = ranking_on(&p) ? 1 : 0;
    a.rescore_top = p.rescore_top;
    const int want_pose = r->out.pose != nullptr;
    const int rank_smem = a.ranking ? rank_smem_bytes(a.S) : 0;
    // restart tiles: 4 lanes per restart (the throughput tile) and, for
    // requests that do not rank poses, 16 (every restart of a ligand in
    // flight: a short chain per ligand, one CTA per SM); the option fixes one
    // or lets the worker switch between them by the backlog
    const int lopt = c->serve_loop_lanes.load();
    dl.ntiles = a.ranking ? 1 : 2;
    cudaError_t e;
    for (int t = 0; t < dl.ntiles; ++t) {
        DeviceLoop::Tile &T = dl.tiles[t];
        T.lanes = t == 0 ? kLanesPerRestart : 16;
        int W = t == 0 ? choose_warps(a.S, c->warps_opt.load()) : std::min(16, (a.S + 1) / 2);
        for (;;) {
            T.ly = make_layout(dl.nmax, dl.rmax, a.P, W, want_pose);
            T.lrt = make_layout_rt(dl.nmax, dl.rmax, a.P, want_pose, 32 / T.lanes);
            T.smem = std::max(T.ly.cta_bytes + W * T.lrt.warp_bytes, T.ly.cta_bytes + rank_smem);
            if ((e = loop_kernel_attributes(W, T.smem, &T.occ, a.ranking, a.rigid_steps > 0, T.lanes)) != cudaSuccess)
                return fail(LG_ECUDA, std::string("serving loop kernel attributes: ") + cudaGetErrorString(e));
            if (T.occ > 0 || W == 1) break;
            W = std::max(1, W / 2);
        }
        if (T.occ <= 0) return fail(LG_EINVAL, "serving loop kernel does not fit on an SM");
        T.W = W;
        T.grid = ctx_num_sms(c) * T.occ;
    }
    dl.adaptive = dl.ntiles == 2 && lopt == 0;
    dl.low_since = -1.0;
    loop_apply_tile(dl, dl.ntiles == 2 && lopt != kLanesPerRestart ? 1 : 0);
    dl.held_n = std::max(dl.tiles[0].grid, dl.ntiles == 2 ? dl.tiles[1].grid : 0);
    // one entry per CTA of the widest tile: centroid, subtree ends and, with
    // ranking, a pose slot
    const int slots = a.ranking ? dl.held_n : 0;
    if (dl.scratch.ensure(scratch_bytes(dl.held_n, dl.rmax, slots, a.S, a.P, a.ly.nmax)))
        return fail(LG_ENOMEM, "serving loop scratch allocation failed");
    a.scr = carve_scratch(dl.scratch.p, dl.held_n, dl.rmax, slots, a.S, a.P, a.ly.nmax);
    a.scr.per_cta = 1;
    if (dl.held.ensure(8 * (size_t)dl.held_n)) return fail(LG_ENOMEM, "serving loop allocation failed");
    // arenas: 2^18 ligand slots, 2^23 atoms, 2^21 torsional bonds (about 170 MB of
    // device memory), at least twice the request, halved while free memory
    // minus the reserve cannot hold them
    loop_free_arenas(dl);
    size_t CL = 1 << 18, CA = 1 << 23, CR = 1 << 21;
    while (CL < 2 * ((size_t)r->L + 1)) CL <<= 1;
    while (CA < 2 * (size_t)r->A) CA <<= 1;
    while (CR < 2 * (size_t)r->R) CR <<= 1;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const size_t reserve = (size_t)c->serve_reserve_mb << 20;
    auto in_bytes = [](size_t L, size_t A, size_t R) {
        return 3 * al256(4 * L) + al256(8 * L) + 4 * al256(4 * A) + al256(A) + al256(2 * A) + al256(2 * R);
    };
    while (in_bytes(CL, CA, CR) + reserve > fr && CL / 2 >= (size_t)r->L + 1 && CA / 2 >= (size_t)r->A &&
           CR / 2 >= std::max<size_t>((size_t)r->R, 1)) {
        CL /= 2;
        CA /= 2;
        CR /= 2;
    }
    if (dl.arena.ensure(in_bytes(CL, CA, CR))) return fail(LG_ENOMEM, "serving loop arena allocation failed");
    const size_t ob = out_arena_bytes(*r, CL, CA, CR);
    if (cudaHostAlloc(&dl.out, ob, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        dl.out = nullptr;
        return fail(LG_ENOMEM, "serving loop output arena allocation failed");
    }
    dl.cap_l = CL;
    dl.cap_a = CA;
    dl.cap_r = CR;
    {  // device views of the ligand arena
        Carve cv;
        char *b = (char *)dl.arena.p;
        BatchDev &B = a.batch;
        B.L = (int)CL;
        B.atom_off = (const int32_t *)(b + cv.take(4 * CL));
        B.rot_off = (const int32_t *)(b + cv.take(4 * CL));
        B.uid = (const uint64_t *)(b + cv.take(8 * CL));
        B.x = (const float *)(b + cv.take(4 * CA));
        B.y = (const float *)(b + cv.take(4 * CA));
        B.z = (const float *)(b + cv.take(4 * CA));
        B.q = (const float *)(b + cv.take(4 * CA));
        B.type = (const uint8_t *)(b + cv.take(CA));
        B.parent = (const int16_t *)(b + cv.take(2 * CA));
        B.rot_child = (const int16_t *)(b + cv.take(2 * CR));
    }
    {  // host and device views of the output arena
        void *dout = nullptr;
        if ((e = cudaHostGetDevicePointer(&dout, dl.out, 0)) != cudaSuccess)
            return fail(LG_ECUDA, std::string("serving loop output arena: ") + cudaGetErrorString(e));
        const size_t S = r->params.restarts, P = r->params.passes, Rs = r->params.rigid_steps;
        Carve cv;
        lg_dock_result &h = dl.out_h;
        memset(&h, 0, sizeof(h));
        h.mem = LG_MEM_HOST;
        char *hb = (char *)dl.out;
        h.score = (double *)(hb + cv.take(8 * CL));
        h.best_restart = (int32_t *)(hb + cv.take(4 * CL));
        h.status = (int32_t *)(hb + cv.take(4 * CL));
        if (r->out.tors_idx) h.tors_idx = (uint8_t *)(hb + cv.take(P * CR));
        if (r->out.pose) h.pose = (float *)(hb + cv.take(12 * CA));
        if (r->out.restart_score) h.restart_score = (double *)(hb + cv.take(8 * S * CL));
        if (r->out.restart_tors) h.restart_tors = (uint8_t *)(hb + cv.take(S * P * CR));
        if (r->out.rank) h.rank = (int32_t *)(hb + cv.take(4 * S * CL));
        if (r->out.leader) h.leader = (int32_t *)(hb + cv.take(4 * S * CL));
        if (r->out.restart_geo) h.restart_geo = (double *)(hb + cv.take(8 * S * CL));
        if (r->out.restart_rigid) h.restart_rigid = (uint8_t *)(hb + cv.take(S * P * Rs * CL));
        auto dv = [&](const void *hp) -> char * { return hp ? (char *)dout + ((const char *)hp - hb) : nullptr; };
        OutDev &o = a.out;
        o.score = (double *)dv(h.score);
        o.best_restart = (int32_t *)dv(h.best_restart);
        o.status = (int32_t *)dv(h.status);
        o.tors_idx = (uint8_t *)dv(h.tors_idx);
        o.pose = (float *)dv(h.pose);
        o.restart_score = (double *)dv(h.restart_score);
        o.restart_tors = (uint8_t *)dv(h.restart_tors);
        o.rank = (int32_t *)dv(h.rank);
        o.leader = (int32_t *)dv(h.leader);
        o.restart_geo = (double *)dv(h.restart_geo);
        o.restart_rigid = (uint8_t *)dv(h.restart_rigid);
        o.decision_rank = nullptr;
    }
    dl.ra_l.reset(CL);
    dl.ra_a.reset(CA);
    dl.ra_r.reset(CR);
    // an empty ring: no ligand published or claimed, every descriptor invalid
    if ((e = cudaMemsetAsync(dl.d_ctl, 0, sizeof(LoopCtl), dl.feed)) != cudaSuccess ||
        (e = cudaMemsetAsync(dl.d_desc, 0xff, kRing * sizeof(LoopDesc), dl.feed)) != cudaSuccess ||
        (e = cudaMemsetAsync(dl.d_done, 0, 4 * kRing, dl.feed)) != cudaSuccess ||
        (e = cudaMemsetAsync(dl.held.p, 0xff, 8 * (size_t)dl.held_n, dl.feed)) != cudaSuccess ||
        (e = cudaEventRecord(dl.fed, dl.feed)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("serving loop reset: ") + cudaGetErrorString(e));
    memset(dl.h_flags, 0, 8 * kRing);
    dl.next_seq = dl.head = dl.tail = 0;
    dl.held_dirty = false;
    dl.stale = 0;
    // the table starts with the loaded pockets (requests then rarely need a relaunch)
    dl.table.clear();
    {
        std::lock_guard<std::mutex> pg(c->pk_mu);
        for (const PocketDev &pk : c->live_pockets)
            if ((int)dl.table.size() < kLoopPockets) dl.table.push_back(pk);
    }
    dl.table_launched = false;
    dl.kind = r;
    dl.configured = true;
    return LG_OK;
}

// Ligands that CTAs of the ended launches claimed but left undocked, sorted
// ascending into the front of the held array: CTA b of the next launch takes
// held[b], held[b + grid], ... in turn, so the lowest claimed ligands -- the
// first to be published -- are at the front of every CTA's list and no CTA
// waits for a ligand while a lower one sits behind another's (with a grid
// smaller than the last launch's, a CTA drains several).
static cudaError_t loop_sort_held(DeviceLoop &dl) {
    if (!dl.held_dirty) return cudaSuccess;
    std::vector<long long> h((size_t)dl.held_n);
    cudaError_t e = cudaMemcpyAsync(h.data(), dl.held.p, 8 * h.size(), cudaMemcpyDeviceToHost, dl.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(dl.stream);
    if (e != cudaSuccess) return e;
    std::vector<long long> v;
    for (long long x : h)
        if (x >= 0) v.push_back(x);
    std::sort(v.begin(), v.end());
    std::fill(h.begin(), h.end(), -1ll);
    std::copy(v.begin(), v.end(), h.begin());
    e = cudaMemcpyAsync(dl.held.p, h.data(), 8 * h.size(), cudaMemcpyHostToDevice, dl.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(dl.stream);
    return e;
}

static int loop_launch(lg_ctx *c, DeviceLoop &dl) {
    cudaError_t e;
    if ((e = loop_sort_held(dl)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("serving loop held ligands: ") + cudaGetErrorString(e));
    dl.held_dirty = true;
    std::unique_ptr<LoopArgs> la(new LoopArgs());
    memset(la.get(), 0, sizeof(LoopArgs));
    la->ctl = dl.d_ctl;
    la->desc = dl.d_desc;
    la->done = dl.d_done;
    la->flags = dl.d_flags;
    la->held = (long long *)dl.held.p;
    la->held_n = dl.held_n;
    la->ring = kRing;
    la->idle_ns = (uint64_t)c->serve_loop_idle_ms.load() * 1000000ull;
    la->first_seq = dl.head;
    la->np = (int)dl.table.size();
    const lg_dock_params &p = dl.kind->params;
    for (int k = 0; k < la->np; ++k) {
        const PocketDev &pk = dl.table[k];
        const double h = pk.h;
        la->pk[k] = pk;
        la->dc2g[k] = (float)((double)p.d_clash * p.d_clash / (h * h));
        la->thr2g[k] = (float)((double)p.cluster_rmsd * p.cluster_rmsd / (h * h));
        la->rigid_shift_g[k] = (float)((double)p.rigid_shift / h);
    }
    const size_t o_live = offsetof(LoopCtl, live);
    if ((e = cudaStreamWaitEvent(dl.stream, dl.fed, 0)) != cudaSuccess ||
        (e = cudaMemsetAsync((char *)dl.d_ctl + o_live, 0, sizeof(LoopCtl) - o_live, dl.stream)) != cudaSuccess ||
        (e = launch_serve_loop(dl.args, *la, dl.grid, dl.smem, dl.stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dl.h_status, &dl.d_ctl->status, 4, cudaMemcpyDeviceToHost, dl.stream)) != cudaSuccess ||
        (e = cudaEventRecord(dl.ended, dl.stream)) != cudaSuccess)
        return fail(LG_ECUDA, std::string("serving loop launch: ") + cudaGetErrorString(e));
    dl.running = true;
    dl.table_launched = true;
    dl.launches++;
    dl.last_status = -1;
    dl.a_launches = dl.launches;
    dl.a_status = -1;
    return LG_OK;
}

// Whether the launch has ended; records how.
static bool loop_ended(DeviceLoop &dl) {
    if (!dl.running) return true;
    const cudaError_t e = cudaEventQuery(dl.ended);
    if (e == cudaErrorNotReady) return false;
    dl.running = false;
    if (e == cudaSuccess) {
        dl.last_status = *(volatile int32_t *)dl.h_status;
    } else {
        cudaGetLastError();
        dl.last_status = LG_ECUDA;
    }
    dl.a_status = dl.last_status;
    return true;
}

// Ask the launch to stop (its CTAs leave after their current ligand) and wait
// for it; the stop flag is cleared for the next launch.
static void loop_stop(DeviceLoop &dl) {
    if (!dl.running) return;
    cudaMemcpyAsync(&dl.d_ctl->stop, &dl.h_stop[1], 4, cudaMemcpyHostToDevice, dl.feed);
    cudaEventSynchronize(dl.ended);
    loop_ended(dl);
    cudaMemcpyAsync(&dl.d_ctl->stop, &dl.h_stop[0], 4, cudaMemcpyHostToDevice, dl.feed);
    cudaEventRecord(dl.fed, dl.feed);
}

// The table index of a pocket, appended when new (-1: the table is full).
static int loop_pocket(DeviceLoop &dl, const PocketDev &pk) {
    for (int k = 0; k < (int)dl.table.size(); ++k)
        if (dl.table[k].cell_o == pk.cell_o) return k;
    if ((int)dl.table.size() >= kLoopPockets) return -1;
    dl.table.push_back(pk);
    dl.table_launched = false;
    return (int)dl.table.size() - 1;
}

// Publish ring slot rs's request: its ligands into its arena ranges, its
// descriptor (invalidated, body, sequence number), then the published-ligand
// count.
static int loop_publish(DeviceLoop &dl, RingSlot &rs, int pocket) {
    Range range("serve: publish to the device loop");
    const Request &r = *rs.reqs[0];
    const int k = (int)(dl.next_seq % kRing);
    // pinned staging: atom and bond offsets rebased to the arena, then the atom arrays
    const size_t L = r.L, A = r.A, R = r.R;
    Carve cv;
    const size_t o_ao = cv.take(4 * (L + 1)), o_ro = cv.take(4 * (L + 1)), o_uid = cv.take(8 * L);
    const size_t o_x = cv.take(4 * A), o_y = cv.take(4 * A), o_z = cv.take(4 * A), o_q = cv.take(4 * A);
    const size_t o_t = cv.take(A), o_p = cv.take(2 * A), o_rc = cv.take(2 * std::max<size_t>(R, 1));
    if (pinned_get(dl, rs.hin, cv.off)) return fail(LG_ENOMEM, "pinned staging allocation failed");
    char *h = (char *)rs.hin.p;
    int32_t *ao = (int32_t *)(h + o_ao), *ro = (int32_t *)(h + o_ro);
    for (size_t l = 0; l <= L; ++l) {
        ao[l] = (int32_t)(rs.atom + (size_t)r.atom_off[l]);
        ro[l] = (int32_t)(rs.tor + (size_t)r.rot_off[l]);
    }
    memcpy(h + o_uid, r.uid.data(), 8 * L);
    memcpy(h + o_x, r.x.data(), 4 * A);
    memcpy(h + o_y, r.y.data(), 4 * A);
    memcpy(h + o_z, r.z.data(), 4 * A);
    memcpy(h + o_q, r.q.data(), 4 * A);
    memcpy(h + o_t, r.type.data(), A);
    memcpy(h + o_p, r.parent.data(), 2 * A);
    if (R) memcpy(h + o_rc, r.rot_child.data(), 2 * R);
    const BatchDev &B = dl.args.batch;
    cudaError_t e = cudaSuccess;
    auto up = [&](const void *dst, size_t off, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(const_cast<void *>(dst), h + off, n, cudaMemcpyHostToDevice, dl.feed);
    };
    up(B.atom_off + rs.slot, o_ao, 4 * (L + 1));
    up(B.rot_off + rs.slot, o_ro, 4 * (L + 1));
    up(B.uid + rs.slot, o_uid, 8 * L);
    up(B.x + rs.atom, o_x, 4 * A);
    up(B.y + rs.atom, o_y, 4 * A);
    up(B.z + rs.atom, o_z, 4 * A);
    up(B.q + rs.atom, o_q, 4 * A);
    up(B.type + rs.atom, o_t, A);
    up(B.parent + rs.atom, o_p, 2 * A);
    up(B.rot_child + rs.tor, o_rc, 2 * R);
    LoopDesc &d = dl.h_desc[k];
    memset(&d, 0, sizeof(d));
    d.seq = dl.next_seq;
    d.first = dl.tail;
    d.L = r.L;
    d.slot = (int32_t)rs.slot;
    d.pocket = pocket;
    dl.h_seq[k] = dl.next_seq;
    dl.h_tail[k] = dl.tail + (uint64_t)r.L;
    LoopDesc *dd = dl.d_desc + k;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dd->seq, dl.h_busy, 8, cudaMemcpyHostToDevice, dl.feed);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char *)dd + 8, (const char *)&d + 8, sizeof(LoopDesc) - 8, cudaMemcpyHostToDevice, dl.feed);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dd->seq, &dl.h_seq[k], 8, cudaMemcpyHostToDevice, dl.feed);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dl.d_ctl->tail, &dl.h_tail[k], 8, cudaMemcpyHostToDevice, dl.feed);
    if (e != cudaSuccess) return fail(LG_ECUDA, std::string("serving loop publish: ") + cudaGetErrorString(e));
    rs.seq = dl.next_seq;
    dl.next_seq++;
    dl.tail += (uint64_t)r.L;
    return LG_OK;
}

// The request's outputs: views of its ranges of the output arena.
static lg_dock_result loop_outputs(const DeviceLoop &dl, const RingSlot &rs) {
    const Request &r = *rs.reqs[0];
    const size_t S = r.params.restarts, P = r.params.passes, Rs = r.params.rigid_steps;
    const lg_dock_result &h = dl.out_h;
    lg_dock_result v = h;
    v.score = h.score + rs.slot;
    v.best_restart = h.best_restart + rs.slot;
    v.status = h.status + rs.slot;
    if (h.tors_idx) v.tors_idx = h.tors_idx + P * rs.tor;
    if (h.pose) v.pose = h.pose + 3 * rs.atom;
    if (h.restart_score) v.restart_score = h.restart_score + S * rs.slot;
    if (h.restart_tors) v.restart_tors = h.restart_tors + S * P * rs.tor;
    if (h.rank) v.rank = h.rank + S * rs.slot;
    if (h.leader) v.leader = h.leader + S * rs.slot;
    if (h.restart_geo) v.restart_geo = h.restart_geo + S * rs.slot;
    if (h.restart_rigid) v.restart_rigid = h.restart_rigid + S * P * Rs * rs.slot;
    return v;
}

// Completed requests (flags raised by the kernel), then the arena ranges and
// descriptors of the oldest completed ones.  Returns whether any finished.
static bool loop_collect(DeviceLoop &dl) {
    bool any = false;
    for (auto &rs : dl.ring) {
        if (!rs.busy) continue;
        if (__atomic_load_n(&dl.h_flags[rs.seq % kRing], __ATOMIC_ACQUIRE) != rs.seq + 1) continue;
        dl.items += rs.reqs[0]->L;
        dl.a_items = dl.items;
        scatter_outputs(loop_outputs(dl, rs), rs.reqs, true);
        rs.reqs.clear();
        rs.busy = false;
        pinned_put(dl, rs.hin);
        any = true;
    }
    const uint64_t h0 = dl.head;
    while (dl.head < dl.next_seq) {
        const RingSlot &rs = dl.ring[dl.head % kRing];
        if (rs.busy && rs.seq == dl.head) break;
        dl.ra_l.release_front();
        dl.ra_a.release_front();
        dl.ra_r.release_front();
        dl.head++;
    }
    if (dl.head != h0) {  // descriptors before head are complete: CTAs need not scan them
        const int k = (int)((dl.head - 1) % kRing);
        dl.h_head[k] = dl.head;
        cudaMemcpyAsync(&dl.d_ctl->head_seq, &dl.h_head[k], 8, cudaMemcpyHostToDevice, dl.feed);
    }
    return any;
}

// Fail every request in flight (the loop cannot finish them); the next
// request sets the loop up afresh.
static void loop_fail_all(DeviceLoop &dl) {
    for (auto &rs : dl.ring) {
        if (!rs.busy) continue;
        for (auto &q : rs.reqs) {
            q->state = LG_REQ_FAILED;
            q->t_done = now_s();
        }
        rs.reqs.clear();
        rs.busy = false;
        pinned_put(dl, rs.hin);
    }
    dl.head = dl.next_seq;
    dl.configured = false;
}

static void loop_release(DeviceLoop &dl) {
    if (!dl.ready) return;
    loop_stop(dl);
    cudaStreamSynchronize(dl.feed);
    for (auto &rs : dl.ring) rs.hin.release();
    for (auto &kv : dl.spare) cudaFreeHost(kv.second);
    dl.spare.clear();
    loop_free_arenas(dl);
    dl.scratch.release();
    dl.ctl.release();
    dl.held.release();
    if (dl.host) cudaFreeHost(dl.host);
    cudaStreamDestroy(dl.stream);
    cudaStreamDestroy(dl.feed);
    cudaEventDestroy(dl.ended);
    cudaEventDestroy(dl.fed);
    dl.ready = false;
}

static void worker_loop(Server *sv) {
    lg_ctx *c = sv->ctx;
    DeviceLoop &dl = *sv->loop;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (dl.ready && loop_collect(dl)) {
            sv->done_cv.notify_all();
            dl.stale = 0;
        }
        int busy = 0;
        int64_t backlog = 0;
        for (auto &rs : dl.ring)
            if (rs.busy) {
                busy++;
                backlog += rs.reqs.empty() ? 0 : rs.reqs[0]->L;
            }
        loop_ended(dl);
        // the restart tile the backlog asks for: a running launch is stopped
        // (its CTAs leave after their current ligand, claimed ligands carry
        // over) and relaunched below with the other tile
        if (dl.configured && dl.adaptive) {
            const int want = loop_tile_wanted(dl, backlog, now_s());
            if (want != dl.cur) {
                if (dl.running) {
                    lk.unlock();
                    loop_stop(dl);
                    lk.lock();
                }
                loop_apply_tile(dl, want);
                dl.low_since = -1.0;
                dl.a_switches = ++dl.switches;
            }
        }
        if (!dl.running && busy > 0 && dl.last_status != LG_OK && dl.last_status != LG_ETIMEOUT &&
            dl.last_status != -1) {
            // the launch ended on an error with requests unfinished
            loop_fail_all(dl);
            sv->done_cv.notify_all();
            busy = 0;
        }
        // admissions, in arrival order
        while (!sv->queue.empty()) {
            std::shared_ptr<Request> r = sv->queue.front();
            if (!dl.ready && loop_setup(c, dl) != LG_OK) {  // no loop: every queued request fails
                for (auto &q : sv->queue) {
                    q->state = LG_REQ_FAILED;
                    q->t_done = now_s();
                }
                sv->queue.clear();
                sv->done_cv.notify_all();
                break;
            }
            if (!loop_fits(dl, *r)) {
                if (busy > 0) break;  // the running kind drains first
                lk.unlock();
                loop_stop(dl);
                lk.lock();
                if (loop_configure(c, dl, r) != LG_OK) {
                    sv->queue.pop_front();
                    r->state = LG_REQ_FAILED;
                    r->t_done = now_s();
                    sv->done_cv.notify_all();
                    continue;
                }
            }
            int pocket = loop_pocket(dl, r->pocket);
            if (pocket < 0) {  // the table is full: drain, then a fresh table
                if (busy > 0) break;
                lk.unlock();
                loop_stop(dl);
                lk.lock();
                dl.table.clear();
                pocket = loop_pocket(dl, r->pocket);
            }
            RingSlot &rs = dl.ring[dl.next_seq % kRing];
            if (rs.busy) break;  // ring full
            // room in the arenas (released in admission order as requests finish)
            size_t s_at = 0, a_at = 0, t_at = 0;
            const RingAlloc::Mark ml = dl.ra_l.mark(), ma = dl.ra_a.mark();
            if (!dl.ra_l.alloc((size_t)r->L + 1, &s_at)) break;
            if (!dl.ra_a.alloc((size_t)r->A, &a_at)) {
                dl.ra_l.rollback(ml);
                break;
            }
            if (!dl.ra_r.alloc((size_t)r->R, &t_at)) {
                dl.ra_l.rollback(ml);
                dl.ra_a.rollback(ma);
                break;
            }
            sv->queue.pop_front();
            r->state = LG_REQ_RUNNING;
            rs.busy = true;
            rs.reqs.assign(1, r);
            rs.slot = s_at;
            rs.atom = a_at;
            rs.tor = t_at;
            lk.unlock();
            // a pocket the running launch's table lacks: relaunch with the table
            if (dl.running && !dl.table_launched) loop_stop(dl);
            int rc = loop_publish(dl, rs, pocket);
            if (rc == LG_OK && !dl.running) rc = loop_launch(c, dl);
            lk.lock();
            if (rc != LG_OK) {
                // the ranges stay reserved (released in order); the request fails
                rs.busy = false;
                pinned_put(dl, rs.hin);
                for (auto &q : rs.reqs) {
                    q->state = LG_REQ_FAILED;
                    q->t_done = now_s();
                }
                rs.reqs.clear();
                sv->done_cv.notify_all();
                continue;
            }
            busy++;
        }
        // work left on the device after the launch ended (idle CTAs left
        // while ligands were still being published): launch again
        if (busy > 0 && !dl.running) {
            // a launch that ended idle with requests unfinished has CTAs
            // waiting on ligands that are not published: a request's ligands
            // are all published at admission, so many such launches in a row
            // with no request finishing mean the loop cannot progress
            if (dl.last_status == LG_ETIMEOUT && ++dl.stale > 100) {
                loop_fail_all(dl);
                sv->done_cv.notify_all();
                dl.stale = 0;
                continue;
            }
            lk.unlock();
            const int rc = loop_launch(c, dl);
            lk.lock();
            if (rc != LG_OK) {
                loop_fail_all(dl);
                sv->done_cv.notify_all();
                busy = 0;
            }
        }
        if (sv->stop && sv->queue.empty() && busy == 0) break;
        if (busy > 0)
            sv->cv.wait_for(lk, std::chrono::microseconds(50));
        else if (dl.running)
            sv->cv.wait_for(lk, std::chrono::milliseconds(1));
        else if (sv->queue.empty() && !sv->stop)
            sv->cv.wait(lk);
    }
    lk.unlock();
    loop_release(dl);
}

static Server *get_server(lg_ctx *c) {
    std::lock_guard<std::mutex> g(c->serve_mu);
    if (c->server) return c->server;
    Server *sv = new Server();
    sv->ctx = c;
    cudaSetDevice(c->device);
    if (c->serve_device_loop) {
        sv->loop = new DeviceLoop();
        sv->th = std::thread(worker_loop, sv);
    } else {
        sv->slots.resize(c->serve_max_inflight);
        for (auto &sl : sv->slots) {
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        }
        sv->th = std::thread(worker, sv);
    }
    c->server = sv;
    return sv;
}

void serve_stats(lg_ctx *c, lg_stats *st) {
    std::lock_guard<std::mutex> g(c->serve_mu);
    const Server *sv = c->server;
    if (!sv || !sv->loop) return;
    st->serve_loop_status = sv->loop->a_status.load();
    st->serve_loop_launches = sv->loop->a_launches.load();
    st->serve_loop_items = sv->loop->a_items.load();
    st->serve_loop_switches = sv->loop->a_switches.load();
}

void serve_stop(lg_ctx *c) {
    Server *sv;
    {
        std::lock_guard<std::mutex> g(c->serve_mu);
        sv = c->server;
        c->server = nullptr;
    }
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
        // queued requests that never reached the device fail
        for (auto &r : sv->queue) {
            r->state = LG_REQ_FAILED;
            r->t_done = now_s();
        }
        sv->queue.clear();
    }
    sv->cv.notify_all();
    sv->th.join();
    sv->done_cv.notify_all();
    delete sv->loop;  // released by its worker
    for (auto &sl : sv->slots) {
        sl.in.release();
        sl.out.release();
        sl.scratch.release();
        sl.lp.release();
        sl.hin.release();
        sl.hout.release();
        sl.hlp.release();
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
    }
    delete sv;
}

}  // namespace lg

using namespace lg;

extern "C" {

int lg_stream_submit(lg_ctx *c, int32_t pid, const lg_ligand_batch *b, const lg_dock_params *p, lg_dock_result *o,
                     uint64_t *ticket) {
    if (!c || !b || !p || !o || !ticket) return fail(LG_EINVAL, "null argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (b->mem != LG_MEM_HOST || o->mem != LG_MEM_HOST) return fail(LG_EINVAL, "serving takes host memory");
    if (b->L < 0) return fail(LG_EINVAL, "L must be >= 0");
    if (b->L > 0 && (!b->atom_off || !b->x || !b->y || !b->z || !b->q || !b->type || !b->parent || !b->rot_off || !b->uid))
        return fail(LG_EINVAL, "null batch array");
    if (!o->score || !o->best_restart || !o->status) return fail(LG_EINVAL, "score, best_restart and status are required");
    if (o->decision_rank) return fail(LG_EINVAL, "decision_rank is not served (use lg_dock_batch)");
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (pid < 0 || pid >= (int)c->pockets.size() || !c->pockets[pid].live) return fail(LG_ENOPOCKET, "unknown pocket");
        r->pocket = c->pockets[pid].dev;
    }
    r->params = *p;
    r->out = *o;
    r->L = b->L;
    if (b->L > 0) {
        if ((rc = host_batch_shape(b, &r->A, &r->R, &r->nmax, &r->rmax))) return rc;
        if (r->R > 0 && !b->rot_child) return fail(LG_EINVAL, "null rot_child");
        if (p->max_atoms > 0) r->nmax = std::min(r->nmax, p->max_atoms);
        if (p->max_rot > 0) r->rmax = std::min(r->rmax, p->max_rot);
        r->atom_off.assign(b->atom_off, b->atom_off + b->L + 1);
        r->rot_off.assign(b->rot_off, b->rot_off + b->L + 1);
        r->uid.assign(b->uid, b->uid + b->L);
        r->x.assign(b->x, b->x + r->A);
        r->y.assign(b->y, b->y + r->A);
        r->z.assign(b->z, b->z + r->A);
        r->q.assign(b->q, b->q + r->A);
        r->type.assign(b->type, b->type + r->A);
        r->parent.assign(b->parent, b->parent + r->A);
        if (r->R) r->rot_child.assign(b->rot_child, b->rot_child + r->R);
    }
    Server *sv = get_server(c);
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->queue.size() >= Server::kMaxQueued) return fail(LG_EAGAIN, "serving queue full");
        r->ticket = sv->next_ticket++;
        r->t_submit = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        if (r->L == 0) {
            r->state = LG_REQ_DONE;
            r->t_done = r->t_submit;
        } else {
            sv->queue.push_back(r);
        }
        sv->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    sv->cv.notify_one();
    return LG_OK;
}

int lg_stream_poll(lg_ctx *c, uint64_t ticket, int32_t *state, double *latency) {
    if (!c || !state) return fail(LG_EINVAL, "null argument");
    Server *sv = get_server(c);
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(LG_EINVAL, "unknown ticket");
    *state = it->second->state;
    if (latency) *latency = it->second->state >= LG_REQ_DONE ? it->second->t_done - it->second->t_submit : -1.0;
    return LG_OK;
}

int lg_stream_wait(lg_ctx *c, uint64_t ticket, int32_t timeout_ms) {
    if (!c) return fail(LG_EINVAL, "null argument");
    Server *sv = get_server(c);
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(LG_EINVAL, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    const bool ok = sv->done_cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                         [&] { return r->state >= LG_REQ_DONE; });
    if (!ok) return fail(LG_ETIMEOUT, "request not finished within the timeout");
    if (r->state == LG_REQ_FAILED) return fail(LG_ECUDA, "request failed");
    return LG_OK;
}

}  // extern "C"
