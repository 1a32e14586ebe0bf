// Context state of liblgdock (host side).  Internal; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lg_internal.h"

namespace lg {

// Named NVTX range around a host-side phase, for timeline profilers (a no-op
// unless a tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t n);  // grow-only; 0 on success
    void release();
};

// Carves aligned sub-arrays out of one allocation.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    }
};

// Device image of a host batch: byte offsets of its arrays and its size.
struct BatchImage {
    size_t o_aoff, o_roff, o_uid, o_x, o_y, o_z, o_q, o_t, o_p, o_rc, bytes;
    BatchImage(int L, int64_t A, int64_t R) {
        Carve c;
        o_aoff = c.take(4 * (size_t)(L + 1));
        o_roff = c.take(4 * (size_t)(L + 1));
        o_uid = c.take(8 * (size_t)L);
        o_x = c.take(4 * (size_t)A);
        o_y = c.take(4 * (size_t)A);
        o_z = c.take(4 * (size_t)A);
        o_q = c.take(4 * (size_t)A);
        o_t = c.take((size_t)A);
        o_p = c.take(2 * (size_t)A);
        o_rc = c.take(2 * (size_t)std::max<int64_t>(R, 1));
        bytes = c.off;
    }
};

struct PocketRec {
    bool live = false;
    PocketDev dev{};
    void *mem = nullptr;
    size_t bytes = 0;
};

struct Server;  // lg_serve.cu

int fail(int code, const std::string &msg);
bool ranking_on(const lg_dock_params *p);
int check_params(const lg_dock_params *p);
int host_batch_shape(const lg_ligand_batch *b, int64_t *A, int64_t *R, int *nmax, int *rmax);
int stage_batch(DevBuf &buf, const lg_ligand_batch *b, int64_t A, int64_t R, BatchDev *d, cudaStream_t s);
size_t batch_image_bytes(int L, int64_t A, int64_t R);
int upload_batch(void *dev, const lg_ligand_batch *b, int64_t A, int64_t R, BatchDev *d, cudaStream_t s);
void serve_stats(lg_ctx *c, lg_stats *st);  // the serving loop's figures (lg_get_stats)
int stage_out(DevBuf &buf, const lg_dock_result *o, int L, int S, int P, int64_t A, int64_t R, int Rs, OutDev *d);
int fetch_out(const OutDev &d, const lg_dock_result *o, int L, int S, int P, int64_t A, int64_t R, int Rs,
              cudaStream_t s);
int checks_result(cudaStream_t s);  // a debug build's bounds-check record as the call's error
int dock_device(lg_ctx *ctx, const PocketDev &pk, const BatchDev &bd, const OutDev &od, const lg_dock_params *p,
                int nmax, int rmax, DevBuf &scratch, cudaStream_t s, lg_stats *st, cudaEvent_t *tev,
                const MultiDev *multi = nullptr, unsigned class_mask = (1u << kSizeClasses) - 1,
                bool allow_graph = false, bool reuse_prep = false);
unsigned host_class_mask(const lg_ligand_batch *b);
int resolve_batch(lg_ctx *c, const lg_ligand_batch *b, const lg_dock_params *p, cudaStream_t s, BatchDev *bd,
                  int64_t *A, int64_t *R, int *nmax, int *rmax);
int resolve_out(lg_ctx *c, DevBuf &buf, const lg_ligand_batch *b, const lg_dock_result *o, int S, int P, int Rs,
                cudaStream_t s, int64_t *A, int64_t *R, OutDev *od);
cudaEvent_t *next_timing_events(lg_ctx *c);
void harvest_timing(lg_ctx *c);
void serve_stop(lg_ctx *c);
int choose_warps(int S, int opt, int lanes = kLanesPerRestart);
void l2_window_of(lg_ctx *c, const PocketDev &pk, const void **base, size_t *bytes, float *hit);

}  // namespace lg

struct lg_ctx {
    int device = 0;
    int num_sms = 0;
    std::mutex mu;  // serialises the calls that use the context's own buffers
    std::vector<lg::PocketRec> pockets;
    lg::DevBuf in_buf, out_buf, scratch;
    std::vector<cudaStream_t> plain_streams;
    std::vector<cudaEvent_t> join_events;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // plain-mode fork (others unused)
    bool timing = false;
    lg_stats stats{};
    // timing ring: (start, end) event pairs of calls not yet harvested
    static constexpr int kTimingRing = 64;
    cudaEvent_t tev[kTimingRing][2] = {};
    int tev_head = 0, tev_pending = 0;
    // options read by the serving worker too (lg_set_option writes them)
    std::atomic<int> warps_opt{0};
    std::atomic<int> lanes_opt{0};  // lanes per restart of batched launches (0: tuned or chosen)
    int serve_max_inflight = 8;  // read when the server starts
    bool serve_device_loop = true;    // read when the server starts: the device-resident loop serves requests
    std::atomic<int> serve_loop_idle_ms{100};  // idle limit of the loop's CTAs
    std::atomic<int> serve_loop_lanes{0};      // the loop's restart tile: 4 or 16 lanes per restart, 0 by the backlog
    std::atomic<int> serve_max_merge{4096};        // ligands per merged batch
    std::atomic<bool> serve_cross_pocket{false};   // merge requests aimed at different pockets
    int64_t serve_reserve_mb = 1024;
    std::mutex serve_mu;  // guards `server` creation
    lg::Server *server = nullptr;
    // several pockets in one launch (lg_dock_multi)
    std::vector<lg::DevBuf> multi_out;
    // autotuner: restart tile (lanes per restart) and warps per CTA chosen by
    // timing, per (size class, restarts, passes, atoms, torsions, features) of
    // the batched kernel
    std::atomic<bool> autotune{true};
    std::atomic<bool> size_classes{true};  // one batched launch per size class when the atom maximum exceeds 64
    // captured CUDA graphs of device-resident lg_dock_batch calls (most recent
    // last); graphs: 0 off, 1 capture a call's arguments on first sight, 2
    // capture them when they recur (graph_seen: recent calls' arguments)
    std::atomic<int> graphs{2};
    std::vector<std::vector<char>> graph_seen;
    struct GraphRec {
        std::vector<char> key;
        cudaGraphExec_t exec = nullptr;
        int launches = 0;
    };
    std::vector<GraphRec> graph_cache;
    std::mutex tune_mu;
    std::map<std::array<int, 8>, std::pair<int, int>> tune;  // key -> (lanes per restart, warps per CTA)
    lg::DevBuf flat_buf;  // lg_flatten_batch: host-output staging and the preparation's unused outputs
    int multi_pocket_major = 1;
    bool pack_host = false;  // lg_pocket_load packs the cells on the host (else on the device)
    // L2 residency of the pockets: the persisting set-aside (process-local
    // context limit, sized for the largest loaded pocket's overlap cells) and
    // the device's limits; the docking launches mark their pocket's overlap
    // cells persisting through an access-policy window (option "l2_window")
    size_t l2_persist_max = 0, l2_window_max = 0;
    size_t l2_persist_prev = 0;  // the limit found at creation, restored at destruction
    size_t l2_persist_set = 0;   // the set-aside this context asked for (0: none)
    std::atomic<bool> l2_window{true};
    // the loaded pockets, for the serving loop's pocket table (its worker
    // does not take `mu`)
    std::mutex pk_mu;
    std::vector<lg::PocketDev> live_pockets;
    // orders the calls that share `scratch` (and `flat_buf`) on the device: a
    // call's stream waits for the previous such call's work to finish
    cudaEvent_t scratch_ev = nullptr;
    // size classes launched side by side: the classes after the first run on
    // these streams, forked from and joined back into the call's stream
    // (class_mu held while a call enqueues on them)
    std::mutex class_mu;
    cudaStream_t class_streams[2] = {};
    cudaEvent_t class_fork = nullptr, class_join[2] = {};
};

namespace lg {

inline int ctx_num_sms(lg_ctx *c) { return c->num_sms; }
// Bracket the device work of a call that uses the context's scratch buffers.
inline cudaError_t scratch_acquire(lg_ctx *c, cudaStream_t s) { return cudaStreamWaitEvent(s, c->scratch_ev, 0); }
inline cudaError_t scratch_release(lg_ctx *c, cudaStream_t s) { return cudaEventRecord(c->scratch_ev, s); }
inline int ctx_warps_opt(lg_ctx *c) { return c->warps_opt; }
inline bool ctx_timing(lg_ctx *c) { return c->timing; }
inline cudaEvent_t ctx_event(lg_ctx *c, int i) { return c->ev[i]; }
inline std::vector<cudaStream_t> &ctx_streams(lg_ctx *c) { return c->plain_streams; }
inline cudaEvent_t ctx_join_event(lg_ctx *c, int i) { return c->join_events[i]; }
inline int ctx_plain_streams(lg_ctx *c, int n) {
    while ((int)c->plain_streams.size() < n) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(s);
            return -1;
        }
        c->plain_streams.push_back(s);
        c->join_events.push_back(e);
    }
    return 0;
}

// Create the context's size-class streams and events on first use (class_mu held).
inline int ctx_class_streams(lg_ctx *c) {
    if (c->class_fork) return 0;
    for (int i = 0; i < 2; ++i) {
        if (!c->class_streams[i] && cudaStreamCreateWithFlags(&c->class_streams[i], cudaStreamNonBlocking) != cudaSuccess)
            return -1;
        if (!c->class_join[i] && cudaEventCreateWithFlags(&c->class_join[i], cudaEventDisableTiming) != cudaSuccess)
            return -1;
    }
    return cudaEventCreateWithFlags(&c->class_fork, cudaEventDisableTiming) == cudaSuccess ? 0 : -1;
}

}  // namespace lg
