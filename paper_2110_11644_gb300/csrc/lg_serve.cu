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
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

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

struct Server {
    lg_ctx *ctx = nullptr;
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
    // pinned input image: CSR arrays of the merged batch
    const size_t bytes_in = 8 * (size_t)(L + 1) + 8 * (size_t)L + 19 * (size_t)A + 2 * (size_t)R + 64;
    if (sl.hin.ensure(bytes_in)) return fail(LG_ENOMEM, "pinned staging allocation failed");
    char *h = (char *)sl.hin.p;
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
    for (auto &r : sl.reqs) {
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
    lg_ligand_batch mb{};
    mb.L = L;
    mb.mem = LG_MEM_HOST;
    mb.atom_off = aoff;
    mb.rot_off = roff;
    mb.uid = uid;
    mb.x = x; mb.y = y; mb.z = z; mb.q = q;
    mb.type = ty;
    mb.parent = par;
    mb.rot_child = rc;
    // pinned output image
    lg_dock_result &hr = sl.hres;
    memset(&hr, 0, sizeof(hr));
    hr.mem = LG_MEM_HOST;
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
    if (sl.hout.ensure(ob + 64)) return fail(LG_ENOMEM, "pinned result allocation failed");
    char *o = (char *)sl.hout.p;
    hr.score = (double *)o; o += 8 * (size_t)L;
    if (want_rs) { hr.restart_score = (double *)o; o += 8 * (size_t)L * S; }
    if (want_g) { hr.restart_geo = (double *)o; o += 8 * (size_t)L * S; }
    hr.best_restart = (int32_t *)o; o += 4 * (size_t)L;
    hr.status = (int32_t *)o; o += 4 * (size_t)L;
    if (want_rk) { hr.rank = (int32_t *)o; o += 4 * (size_t)L * S; }
    if (want_ld) { hr.leader = (int32_t *)o; o += 4 * (size_t)L * S; }
    if (want_p) { hr.pose = (float *)o; o += 12 * (size_t)A; }
    if (want_t) { hr.tors_idx = (uint8_t *)o; o += (size_t)P * R; }
    if (want_rt) { hr.restart_tors = (uint8_t *)o; o += (size_t)S * P * R; }
    if (want_rg) { hr.restart_rigid = (uint8_t *)o; }

    cudaSetDevice(c->device);
    BatchDev bd;
    OutDev od;
    int rc2;
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

// Split the merged results back into each request's output buffers.
static void finish_slot(Slot &sl, bool ok) {
    const lg_dock_result &hr = sl.hres;
    int l0 = 0;
    int64_t a0 = 0, k0 = 0;
    const double t = now_s();
    for (auto &r : sl.reqs) {
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

static Server *get_server(lg_ctx *c) {
    std::lock_guard<std::mutex> g(c->serve_mu);
    if (c->server) return c->server;
    Server *sv = new Server();
    sv->ctx = c;
    cudaSetDevice(c->device);
    sv->slots.resize(c->serve_max_inflight);
    for (auto &sl : sv->slots) {
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    sv->th = std::thread(worker, sv);
    c->server = sv;
    return sv;
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
