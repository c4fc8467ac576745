// pt_serve.cu -- continuous batching of PT-QMC requests.
//
// Requests arrive at any time (pt_server_submit) and wait in a FIFO until a slot and room
// in a preallocated device arena are free; then their data and initial state are placed
// in the arena, where their spins, (E, M), rung permutation, statistics and sweep / pass
// counters stay until they finish. Every pt_server_step is one launch in which each
// admitted request advances by up to `quantum` sweeps (whole swap intervals), so the work
// of requests that arrived at different times overlaps on the device; requests that
// complete are reported and admission runs again.
//
// Default (streamed) mode: every admitted request is launched at once, with all of its
// sweeps, on one stream of a pool -- one CTA per chain, the launch plan pt_create would
// choose -- and its completion is tracked with an event. Requests that arrive while others
// run start as soon as a slot, arena room and the in-flight chain budget allow, and the
// GPU runs their kernels side by side as SMs become free, so the device does the
// continuous batching at CTA granularity. A backlog (kGroupMin or more waiting requests)
// starts together in one persistent batched launch, which packs chains onto clusters and
// sustains a higher rate under overload. Stepped mode (pt_server_options.reserved[1] = 1) instead advances all
// admitted requests by a quantum of sweeps per launch, one CTA per chain when they all fit
// (wide), chains packed onto clusters otherwise (packed).
// A request's arithmetic never depends on what else runs or on the launch shape: its
// result equals pt_create + pt_run on it alone.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <map>
#include <vector>

#include "pt.h"
#include "pt_internal.h"

using namespace ptq;

namespace {

// First-fit allocator over [0, size) of the device arena, 256-byte granules.
class ArenaAllocator {
   public:
    explicit ArenaAllocator(size_t size) : size_(size) { free_.push_back({0, size}); }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (size_t k = 0; k < free_.size(); ++k) {
            if (free_[k].size >= bytes) {
                *off = free_[k].off;
                free_[k].off += bytes;
                free_[k].size -= bytes;
                if (free_[k].size == 0) free_.erase(free_.begin() + k);
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = std::lower_bound(free_.begin(), free_.end(), off,
                                   [](const Range& r, size_t o) { return r.off < o; });
        it = free_.insert(it, {off, bytes});
        // merge with the next and the previous free range
        if (it + 1 != free_.end() && it->off + it->size == (it + 1)->off) {
            it->size += (it + 1)->size;
            free_.erase(it + 1);
        }
        if (it != free_.begin() && (it - 1)->off + (it - 1)->size == it->off) {
            (it - 1)->size += it->size;
            free_.erase(it);
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

   private:
    struct Range {
        size_t off, size;
    };
    std::vector<Range> free_;
    size_t size_, used_ = 0;
};

// Requests launched together as one persistent batched launch share a device block holding
// their records, the work order, the work counter and a status word.
// A backlog group: requests admitted together into one persistent batched launch. Each
// member completes on its own (the kernel raises its flag once its chains are written back);
// the group's block (instance records, work counter, flags) is freed once the launch ends.
struct ServeGroup {
    size_t off = 0, bytes = 0, status_off = 0, flags_off = 0;
    int refs = 0;                 // members not yet completed
    int n = 0;
    int token = 0;                // the value a member's flag takes when it is done
    std::vector<int> flags;       // host copy of the members' done flags
    cudaEvent_t done = nullptr;   // the launch's end
    cudaEvent_t zeroed = nullptr; // the block's counter, status and flags are zero (before the launch)
    int stream_idx = 0;           // the pool stream it runs on
    int ctas = 0;                 // CTAs launched (each holds an SM until the launch ends)
};

struct ServeReq {
    int64_t id;
    pt_request req;  // pointers cleared after preparation
    Prepared prep;
    size_t block_off = 0, block_bytes = 0;
    BatchInstance inst;
    int64_t remaining = 0;
    int state = 0;  // 0 queued, 1 on the device, 2 finished
    // streamed mode
    cudaEvent_t done = nullptr;
    int stream_idx = 0;
    ServeGroup* group = nullptr;  // set while the request runs in a batched launch
    int group_index = -1;         // its problem index (and flag) in that launch
};

// Streamed mode launches a request's sweeps in pieces of at most this many swap passes.
constexpr int kStreamedPasses = 256;

// Streamed mode under backlog: once this many requests wait, they start together in one
// persistent batched launch (chains packed onto thread-block clusters), which sustains a
// higher rate than one launch per request. Below it, a request starts on its own launch
// while the SMs it needs are free: a request launched alone is one cooperative launch whose
// chains wait for one another's swap mailboxes, so every one of its CTAs must be resident
// together. Each in-flight chain is counted as one SM (a CTA of the streamed kernel can
// need a whole SM's shared memory), and a running group launch as its CTAs until it ends.
constexpr int kGroupMin = 8;

}  // namespace

struct pt_server {
    cudaStream_t stream;
    bool own_stream;
    unsigned char* arena;
    ArenaAllocator* alloc;
    int max_active, quantum, cluster, threads, n_clusters;
    bool adaptive_cluster;   // backlog launches pick their cluster size from the free SMs
    int ncl_by_log2[5];      // clusters of 1, 2, 4, 8, 16 CTAs that fit at once (0: none)
    int wide_threads, n_sm;
    bool wide;
    MultiProblem* d_multi;
    int2* d_wmap;
    int wmap_capacity;
    int64_t wide_steps;
    bool streamed;
    std::vector<cudaStream_t> pool;
    std::vector<int> stream_load;  // requests launched alone plus groups still running, per stream
    int next_stream;
    long long inflight_sms;  // streamed mode: SMs held by requests launched alone and by group launches
    int64_t group_launches;
    size_t smem_cap;
    std::map<int64_t, ServeReq*> reqs;
    std::deque<int64_t> queued;
    std::vector<int64_t> active;
    std::deque<int64_t> finished_unreported;
    std::vector<ServeGroup*> retiring;  // groups whose members are all done, launch still running
    int64_t next_id, steps, launches;
    BatchInstance* d_inst;
    int32_t* d_order;
    int* d_counter;
    int* d_status;
    int2* d_map;
    int map_capacity;
    std::vector<void*> allocs;
    int err;
    char msg[256];
};

static thread_local char g_srv_create_msg[256] = "";

static int sfail(pt_server* s, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s ? s->msg : g_srv_create_msg, 256, fmt, ap);
    va_end(ap);
    if (s && (code == PT_ECUDA || code == PT_ETIMEDOUT)) s->err = code;
    return code;
}

static void free_server(pt_server* s) {
    for (cudaStream_t st : s->pool) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    std::vector<ServeGroup*> groups(s->retiring);
    for (auto& kv : s->reqs)
        if (kv.second->group && std::find(groups.begin(), groups.end(), kv.second->group) == groups.end())
            groups.push_back(kv.second->group);
    for (ServeGroup* grp : groups) {
        if (grp->done) cudaEventDestroy(grp->done);
        if (grp->zeroed) cudaEventDestroy(grp->zeroed);
        delete grp;
    }
    for (auto& kv : s->reqs) {
        if (kv.second->done) cudaEventDestroy(kv.second->done);
        delete kv.second;
    }
    for (void* p : s->allocs) cudaFree(p);
    delete s->alloc;
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" int pt_server_create(const pt_server_options* opt, void* cuda_stream, pt_server** out) {
    if (!out) return sfail(nullptr, PT_EINVAL, "null output");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return sfail(nullptr, PT_ENODEV, "no CUDA device");
    pt_server* s = new pt_server();
    s->stream = (cudaStream_t)cuda_stream;
    s->own_stream = false;
    s->arena = nullptr;
    s->alloc = nullptr;
    s->next_id = 1;
    s->steps = s->launches = 0;
    s->err = 0;
    s->msg[0] = 0;
    s->max_active = (opt && opt->max_active > 0) ? opt->max_active : 512;
    s->quantum = (opt && opt->quantum_sweeps > 0) ? opt->quantum_sweeps : 100;
    s->cluster = (opt && opt->cluster_size > 0) ? opt->cluster_size : 2;
    s->adaptive_cluster = !(opt && opt->cluster_size > 0);
    s->threads = 512;
    s->wide_threads = 256;
    s->wide = !(opt && opt->reserved[0] == 1);    // reserved[0] == 1: stepped, packed launches only
    s->streamed = !(opt && (opt->reserved[1] == 1 || opt->reserved[0] == 1));  // reserved[1] == 1: stepped
    s->next_stream = 0;
    s->wide_steps = 0;
    s->inflight_sms = 0;
    s->group_launches = 0;
    if (s->cluster > 16 || s->max_active > 65536) {
        delete s;
        return sfail(nullptr, PT_EINVAL, "cluster_size <= 16 and max_active <= 65536");
    }
    if (!s->stream) {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return sfail(nullptr, PT_ECUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t arena_bytes = (opt && opt->arena_bytes > 0) ? (size_t)opt->arena_bytes : free_b / 2;
    arena_bytes &= ~(size_t)255;
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
    s->smem_cap = (size_t)max_smem - 1024;
    s->map_capacity = 1 << 16;
    s->wmap_capacity = s->n_sm * 8;
    cudaError_t e;
    auto grab = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        s->allocs.push_back(q);
        return q;
    };
    s->arena = (unsigned char*)grab(arena_bytes);
    s->d_inst = (BatchInstance*)grab(sizeof(BatchInstance) * s->max_active);
    s->d_order = (int32_t*)grab(sizeof(int32_t) * s->max_active);
    s->d_counter = (int*)grab(16);
    s->d_status = (int*)grab(16);
    s->d_map = (int2*)grab(sizeof(int2) * s->map_capacity);
    s->d_multi = (MultiProblem*)grab(sizeof(MultiProblem) * s->max_active);
    s->d_wmap = (int2*)grab(sizeof(int2) * s->wmap_capacity);
    if (!s->arena || !s->d_inst || !s->d_order || !s->d_counter || !s->d_status || !s->d_map || !s->d_multi ||
        !s->d_wmap) {
        free_server(s);
        return sfail(nullptr, PT_ENOMEM, "could not allocate the serving arena (%zu bytes)", arena_bytes);
    }
    s->alloc = new ArenaAllocator(arena_bytes);
    if ((e = cudaMemsetAsync(s->d_status, 0, 16, s->stream)) != cudaSuccess) {
        free_server(s);
        return sfail(nullptr, PT_ECUDA, "%s", cudaGetErrorString(e));
    }
    int ncl = 0;
    if ((e = batch_max_clusters(s->cluster, s->threads, s->smem_cap, &ncl)) != cudaSuccess || ncl < 1) {
        free_server(s);
        return sfail(nullptr, PT_EINVAL, "no cluster of %d CTAs fits (%s)", s->cluster, cudaGetErrorString(e));
    }
    s->n_clusters = ncl;
    for (int l = 0; l < 5; ++l) {
        int n = 0;
        if (batch_max_clusters(1 << l, s->threads, s->smem_cap, &n) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 0;
        }
        s->ncl_by_log2[l] = n;
    }
    if (s->streamed) {
        for (int k = 0; k < 16; ++k) {
            cudaStream_t st;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                free_server(s);
                return sfail(nullptr, PT_ECUDA, "cudaStreamCreate failed");
            }
            s->pool.push_back(st);
        }
    }
    *out = s;
    return PT_OK;
}

extern "C" int pt_server_submit(pt_server* s, const pt_request* r, int64_t* id) {
    if (!s || !r || !id) return PT_EINVAL;
    if (s->err) return s->err;
    ServeReq* q = new ServeReq();
    char why[200];
    // levels balanced for the one-CTA-per-chain kernel of a streamed launch (384 consumer
    // threads over the power-of-two word columns of an item); any valid schedule serves
    // the batched kernel of a backlog launch as well
    int cols = 1;
    while (cols < r->P / 8) cols <<= 1;
    const int rc = prepare_request(*r, q->prep, why, sizeof(why), r->P >= 8 ? std::max(1, 384 / cols) : 0);
    if (rc) {
        delete q;
        return sfail(s, rc, "%s", why);
    }
    // mailboxes for the wide launch shape: one entry per rung per swap pass of a step
    q->block_bytes = request_block_layout(q->prep, (size_t)std::max(s->quantum, kStreamedPasses) * q->prep.R);
    if (q->block_bytes > s->alloc->size()) {
        delete q;
        return sfail(s, PT_ENOMEM, "request needs %zu bytes, the arena holds %zu", q->block_bytes, s->alloc->size());
    }
    if (q->prep.R > s->map_capacity) {
        delete q;
        return sfail(s, PT_EINVAL, "too many rungs");
    }
    q->req = *r;
    q->req.inst.ei = q->req.inst.ej = q->req.inst.J = q->req.inst.h = nullptr;
    q->req.ladder = nullptr;
    q->remaining = r->n_sweeps;
    q->id = s->next_id++;
    // the request's shared-memory plan must fit one CTA
    fill_instance(q->inst, q->prep, nullptr, q->req);
    choose_groups(q->inst, s->cluster, s->threads, s->smem_cap);
    if (batch_smem_bytes(q->inst, s->cluster, s->threads) > s->smem_cap) {
        delete q;
        return sfail(s, PT_EINVAL, "request does not fit one CTA's shared memory");
    }
    if (q->prep.sweep_limit < r->n_sweeps) {
        delete q;
        return sfail(s, PT_EOVERFLOW, "request's statistics could overflow int64");
    }
    s->reqs[q->id] = q;
    s->queued.push_back(q->id);
    *id = q->id;
    return PT_OK;
}

// Admit queued requests in arrival order while a slot and arena room are free.
static int admit(pt_server* s) {
    std::vector<ServeReq*> fresh;
    while (!s->queued.empty() && (int)s->active.size() < s->max_active) {
        ServeReq* q = s->reqs[s->queued.front()];
        size_t off = 0;
        if (!s->alloc->alloc(q->block_bytes, &off)) break;
        q->block_off = off;
        unsigned char* base = s->arena + off;
        const Prepared& p = q->prep;
        const int gthreads = q->inst.group_threads, resident = q->inst.resident, thr_res = q->inst.thr_resident;
        fill_instance(q->inst, p, base, q->req);
        q->inst.group_threads = gthreads;
        q->inst.resident = resident;
        q->inst.thr_resident = thr_res;
        std::vector<unsigned char> host(p.off_spins, 0);
        memcpy(&host[p.off_sdesc], p.sdesc.data(), p.sdesc.size() * 4);
        memcpy(&host[p.off_items], p.items.data(), p.items.size() * 4);
        memcpy(&host[p.off_loff], p.level_off.data(), p.level_off.size() * 4);
        memcpy(&host[p.off_thr], p.thr.data(), p.thr.size() * 4);
        memcpy(&host[p.off_coef], p.coef.data(), p.coef.size() * 8);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(base + p.off_spins, 0, q->block_bytes - p.off_spins, s->stream)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "admission upload: %s", cudaGetErrorString(e));
        q->state = 1;
        s->queued.pop_front();
        s->active.push_back(q->id);
        fresh.push_back(q);
    }
    // initial spins and (E, M) of the newly admitted requests, one block per chain
    size_t k = 0;
    while (k < fresh.size()) {
        std::vector<BatchInstance> insts;
        std::vector<int2> map;
        while (k < fresh.size() && (int)insts.size() < s->max_active &&
               (int)(map.size() + fresh[k]->prep.R) <= s->map_capacity) {
            for (int rho = 0; rho < fresh[k]->prep.R; ++rho) map.push_back(make_int2((int)insts.size(), rho));
            insts.push_back(fresh[k]->inst);
            ++k;
        }
        cudaError_t e;
        if ((e = cudaMemcpyAsync(s->d_inst, insts.data(), insts.size() * sizeof(BatchInstance),
                                 cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->d_map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                 s->stream)) != cudaSuccess ||
            (e = launch_batch_init(s->d_inst, s->d_map, (int)map.size(), s->stream)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "admission init: %s", cudaGetErrorString(e));
        s->launches += 1;
    }
    return PT_OK;
}

// Streamed mode: place a request in the arena and launch all of its sweeps on a pool stream.
// A newly admitted request's constants, zeroed state and initial spins, on stream st.
static int upload_request(pt_server* s, ServeReq* q, cudaStream_t st) {
    unsigned char* base = s->arena + q->block_off;
    const Prepared& pr = q->prep;
    const int gthreads = q->inst.group_threads, resident = q->inst.resident, thr_res = q->inst.thr_resident;
    fill_instance(q->inst, pr, base, q->req);
    q->inst.group_threads = gthreads;
    q->inst.resident = resident;
    q->inst.thr_resident = thr_res;
    std::vector<unsigned char> host(pr.off_spins, 0);
    memcpy(&host[pr.off_sdesc], pr.sdesc.data(), pr.sdesc.size() * 4);
    memcpy(&host[pr.off_items], pr.items.data(), pr.items.size() * 4);
    memcpy(&host[pr.off_loff], pr.level_off.data(), pr.level_off.size() * 4);
    memcpy(&host[pr.off_thr], pr.thr.data(), pr.thr.size() * 4);
    memcpy(&host[pr.off_coef], pr.coef.data(), pr.coef.size() * 8);
    std::vector<int2> map(pr.R);
    for (int rho = 0; rho < pr.R; ++rho) map[rho] = make_int2(0, rho);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + pr.off_spins, 0, q->block_bytes - pr.off_spins, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + pr.off_inst, &q->inst, sizeof(BatchInstance), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(base + pr.off_map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = launch_batch_init((const BatchInstance*)(base + pr.off_inst), (const int2*)(base + pr.off_map), pr.R,
                               st)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "streamed admission: %s", cudaGetErrorString(e));
    s->launches += 1;
    return PT_OK;
}

// The pool stream with the least work still running (first such stream from a rotating
// start), so that a new launch never waits in stream order behind a long request or group.
static int pick_stream(pt_server* s) {
    const int n = (int)s->pool.size();
    if ((int)s->stream_load.size() != n) s->stream_load.assign(n, 0);
    int best = s->next_stream;
    for (int k = 0; k < n; ++k) {
        const int i = (s->next_stream + k) % n;
        if (s->stream_load[i] < s->stream_load[best]) best = i;
    }
    s->next_stream = (best + 1) % n;
    s->stream_load[best] += 1;
    return best;
}

static int launch_streamed(pt_server* s, ServeReq* q) {
    q->stream_idx = pick_stream(s);
    cudaStream_t st = s->pool[q->stream_idx];
    int rc = upload_request(s, q, st);
    if (rc) return rc;
    unsigned char* base = s->arena + q->block_off;
    const Prepared& pr = q->prep;
    cudaError_t e;

    // the single-problem packed kernel, as pt_create would plan it
    DevProblem p;
    memset(&p, 0, sizeof(p));
    p.desc = q->inst.sdesc;
    p.items = q->inst.items;
    p.level_off = q->inst.level_off;
    p.thr = q->inst.thr;
    p.coef = q->inst.coef;
    p.spins = q->inst.spins;
    p.E = q->inst.E;
    p.M = q->inst.M;
    p.rung_of_slot = q->inst.rung_of_slot;
    p.slot_of_rung = q->inst.slot_of_rung;
    p.acc = q->inst.acc;
    p.swap_stats = q->inst.swap_stats;
    p.mbox = (Mailbox*)(base + pr.off_mbox);
    p.status = (int*)(base + pr.off_status);
    p.N = pr.N;
    p.P = pr.P;
    p.R = pr.R;
    p.Lmax = pr.Lmax;
    p.nL3 = (2 * pr.Lmax + 1) * 3;
    p.n_levels = pr.n_levels;
    p.dmax = pr.dc;
    p.slot_stride = pr.slot_stride;
    p.withhold_rung = -1;
    p.key0 = q->inst.key0;
    p.key1 = q->inst.key1;
    p.acc_in_smem = (size_t)pr.R * kAccCount * 8 <= 16384 ? 1 : 0;
    p.tables_in_smem = (size_t)pr.R * p.nL3 * 4 <= 49152 ? 1 : 0;
    LaunchPlan plan;
    plan.dclass = pr.dc;
    plan.path = kPathPacked;
    if (sweep_smem_bytes(p, kPathPacked, pr.dc) > s->smem_cap) plan.path = kPathPackedInline;
    if (p.tables_in_smem && sweep_smem_bytes(p, plan.path, pr.dc) > s->smem_cap) p.tables_in_smem = 0;
    if (p.acc_in_smem && sweep_smem_bytes(p, plan.path, pr.dc) > s->smem_cap) p.acc_in_smem = 0;
    plan.smem_bytes = sweep_smem_bytes(p, plan.path, pr.dc);
    if (plan.path == kPathPacked) {
        plan.threads = 512;
        plan.n_consumer = 384;
    } else {
        const long long units = 2ll * pr.N * (pr.P / 8);
        long long avg = (units + pr.n_levels - 1) / pr.n_levels;
        avg = ((avg + 31) / 32) * 32;
        plan.threads = (int)std::min<long long>(512, std::max<long long>(128, avg));
        plan.n_consumer = plan.threads;
    }
    if (prepare_sweep_kernel(plan) != cudaSuccess) return sfail(s, PT_ECUDA, "cudaFuncSetAttribute failed");
    const int sps = q->inst.sweeps_per_swap;
    const bool swaps = sps > 0 && pr.R > 1;
    int per_sm = 0;
    const bool coop = swaps && sweep_kernel_occupancy(p, plan, &per_sm) == cudaSuccess &&
                      (long long)per_sm * s->n_sm >= pr.R;
    long long t = q->inst.t0, qq = q->inst.q0;
    long long left = q->remaining;
    const long long timeout = 5000000000ll;
    if (!swaps || coop) {
        const long long full = swaps ? (left / sps) * sps : 0;
        long long done = 0;
        while (done < left) {
            long long chunk;
            int use_sps = 0;
            if (done < full) {
                chunk = std::min<long long>(full - done, (long long)kStreamedPasses * sps);
                use_sps = sps;
            } else {
                chunk = left - done;
            }
            if ((e = launch_sweeps(p, plan, t, qq, (int)chunk, use_sps, timeout, use_sps > 0, st)) != cudaSuccess)
                return sfail(s, PT_ECUDA, "streamed launch: %s", cudaGetErrorString(e));
            s->launches += 1;
            t += chunk;
            if (use_sps > 0) qq += chunk / sps;
            done += chunk;
        }
        if (!swaps && sps > 0) qq += left / sps;
    } else {
        // chains cannot all be resident: one launch per swap interval and a swap launch
        for (long long done = 0; done + sps <= left; done += sps) {
            if ((e = launch_sweeps(p, plan, t, qq, sps, 0, timeout, false, st)) != cudaSuccess ||
                (e = launch_swap(p, qq, st)) != cudaSuccess)
                return sfail(s, PT_ECUDA, "streamed launch: %s", cudaGetErrorString(e));
            s->launches += 2;
            t += sps;
            qq += 1;
        }
        const long long rest = left % sps;
        if (rest > 0) {
            if ((e = launch_sweeps(p, plan, t, qq, (int)rest, 0, timeout, false, st)) != cudaSuccess)
                return sfail(s, PT_ECUDA, "streamed launch: %s", cudaGetErrorString(e));
            s->launches += 1;
            t += rest;
        }
    }
    if (!q->done && (e = cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    if ((e = cudaEventRecord(q->done, st)) != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    q->inst.t0 = t;
    q->inst.q0 = qq;
    q->remaining = 0;
    q->state = 1;
    return PT_OK;
}

// Requests g, admitted together, in one persistent batched launch on one stream of the pool.
// Returns 1 (nothing launched) when the arena has no room for the group's block.
static int launch_group(pt_server* s, const std::vector<ServeReq*>& g) {
    const int n = (int)g.size();
    // Cluster size: the given one, or the largest of 8, 4 and 2 CTAs at which every member
    // gets a cluster of its own at once (2 when even that is too many). A member runs on one
    // cluster, so a short backlog gets wide clusters (each request's chains over more SMs,
    // lower latency) and a long one narrow clusters (the most requests at once: on this GPU
    // clusters of 2 also sweep the most attempts per second). 16 is not used: fewer of them
    // fit the GPU's SMs, and they lost to 8 on latency as well in measured replays.
    int K = s->cluster, ncl = s->n_clusters;
    if (s->adaptive_cluster) {
        int l = 3;
        while (l > 1 && s->ncl_by_log2[l] < n) --l;
        // every member must fit a CTA of that cluster size (narrower clusters hold more chains
        // per CTA but never need more room than streaming one chain per group)
        for (; l > 1; --l) {
            bool ok = true;
            for (ServeReq* q : g) {
                BatchInstance I = q->inst;
                choose_groups(I, 1 << l, s->threads, s->smem_cap);
                if (batch_smem_bytes(I, 1 << l, s->threads) > s->smem_cap) ok = false;
            }
            if (ok) break;
        }
        K = 1 << l;
        ncl = s->ncl_by_log2[l] > 0 ? s->ncl_by_log2[l] : s->n_clusters;
        if (s->ncl_by_log2[l] <= 0) K = s->cluster;
    }
    ServeGroup* grp = new ServeGroup();
    const size_t order_off = ((size_t)n * sizeof(BatchInstance) + 255) & ~(size_t)255;
    const size_t ctr_off = order_off + (((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255);
    grp->status_off = ctr_off + 16;
    grp->flags_off = ctr_off + 256;
    grp->bytes = grp->flags_off + (((size_t)n * sizeof(int) + 255) & ~(size_t)255);
    grp->n = n;
    grp->flags.assign(n, 0);
    if (!s->alloc->alloc(grp->bytes, &grp->off)) {
        delete grp;
        return 1;
    }
    const int sidx = pick_stream(s);
    cudaStream_t st = s->pool[sidx];
    grp->stream_idx = sidx;
    std::vector<BatchInstance> insts(n);
    size_t smem = 0;
    for (int k = 0; k < n; ++k) {
        ServeReq* q = g[k];
        int rc = upload_request(s, q, st);
        if (rc) return rc;
        q->inst.n_sweeps = (int)q->remaining;
        choose_groups(q->inst, K, s->threads, s->smem_cap);
        smem = std::max(smem, batch_smem_bytes(q->inst, K, s->threads));
        insts[k] = q->inst;
    }
    std::vector<int32_t> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double wx = (double)insts[x].N * insts[x].P * insts[x].R * (double)insts[x].n_sweeps;
        const double wy = (double)insts[y].N * insts[y].P * insts[y].R * (double)insts[y].n_sweeps;
        return wx > wy;
    });
    unsigned char* gb = s->arena + grp->off;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(gb, insts.data(), (size_t)n * sizeof(BatchInstance), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(gb + order_off, order.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemsetAsync(gb + ctr_off, 0, grp->bytes - ctr_off, st)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&grp->zeroed, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(grp->zeroed, st)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "group upload: %s", cudaGetErrorString(e));
    BatchParams bp;
    bp.inst = (BatchInstance*)gb;
    bp.order = (const int32_t*)(gb + order_off);
    bp.count = n;
    bp.next_job = (int*)(gb + ctr_off);
    bp.status = (int*)(gb + grp->status_off);
    bp.done = (int*)(gb + grp->flags_off);
    // a flag left in this arena block by an earlier group (of this server, or of an earlier
    // user of the same device memory) must never match: tokens are unique in the process,
    // and the host reads a group's flags only once the memset above has run (grp->zeroed)
    static std::atomic<unsigned> g_next_token{0};
    grp->token = (int)(g_next_token.fetch_add(1) % 2000000000u) + 1;
    bp.done_token = grp->token;
    if ((e = launch_batch(bp, K, std::min(ncl, n), s->threads, smem, st)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "group launch: %s", cudaGetErrorString(e));
    grp->ctas = std::min(ncl, n) * K;
    s->inflight_sms += grp->ctas;
    if ((e = cudaEventCreateWithFlags(&grp->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(grp->done, st)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    s->launches += 1;
    s->group_launches += 1;
    for (int k = 0; k < n; ++k) {
        ServeReq* q = g[k];
        if (!q->done && (e = cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        if ((e = cudaEventRecord(q->done, st)) != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        q->group_index = k;
        q->stream_idx = sidx;
        q->inst.t0 += q->remaining;
        if (q->inst.sweeps_per_swap > 0) q->inst.q0 += q->remaining / q->inst.sweeps_per_swap;
        q->remaining = 0;
        q->state = 1;
        q->group = grp;
        grp->refs += 1;
    }
    return PT_OK;
}

// Frees the block of a group whose launch has ended (false: still running).
static bool retire_group(pt_server* s, ServeGroup* grp) {
    if (cudaEventQuery(grp->done) != cudaSuccess) return false;
    s->stream_load[grp->stream_idx] -= 1;
    s->inflight_sms -= grp->ctas;
    s->alloc->release(grp->off, grp->bytes);
    cudaEventDestroy(grp->done);
    cudaEventDestroy(grp->zeroed);
    delete grp;
    return true;
}

static int step_streamed(pt_server* s) {
    // groups whose members have all completed: free their blocks once the launch has ended
    {
        std::vector<ServeGroup*> keep;
        for (ServeGroup* grp : s->retiring)
            if (!retire_group(s, grp)) keep.push_back(grp);
        s->retiring.swap(keep);
    }
    // the done flags of the members of groups still running, one small copy per group
    {
        std::vector<ServeGroup*> polled;
        for (int64_t id : s->active) {
            ServeGroup* grp = s->reqs[id]->group;
            if (!grp || std::find(polled.begin(), polled.end(), grp) != polled.end()) continue;
            // the flags are copied on the server's stream, which is not ordered after the
            // group's stream: until the memset that zeroes them has run, the block still holds
            // whatever the memory held before, so they are not read yet
            const cudaError_t z = cudaEventQuery(grp->zeroed);
            if (z == cudaErrorNotReady) continue;
            if (z != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(z));
            polled.push_back(grp);
            const cudaError_t e = cudaMemcpyAsync(grp->flags.data(), s->arena + grp->off + grp->flags_off,
                                                  (size_t)grp->n * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        }
        if (!polled.empty()) {
            const cudaError_t e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        }
    }
    // completions first, so their arena room can go to queued requests
    std::vector<int64_t> still;
    for (int64_t id : s->active) {
        ServeReq* q = s->reqs[id];
        const bool flagged = q->group && q->group->flags[q->group_index] == q->group->token;
        const cudaError_t e = flagged ? cudaSuccess : cudaEventQuery(q->done);
        if (e == cudaErrorNotReady) {
            still.push_back(id);
            continue;
        }
        if (e != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        int st = 0;
        const size_t status_at = q->group ? q->group->off + q->group->status_off : q->block_off + q->prep.off_status;
        const cudaError_t e2 = cudaMemcpy(&st, s->arena + status_at, sizeof(int), cudaMemcpyDeviceToHost);
        if (e2 != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e2));
        if (st == PT_ETIMEDOUT) return sfail(s, PT_ETIMEDOUT, "a swap wait timed out");
        if (st) return sfail(s, PT_ECUDA, "device status %d", st);
        if (!q->group) s->stream_load[q->stream_idx] -= 1;  // its own launch has ended
        if (q->group && --q->group->refs == 0 && !retire_group(s, q->group)) s->retiring.push_back(q->group);
        if (!q->group) s->inflight_sms -= q->prep.R;
        q->group = nullptr;
        q->group_index = -1;
        q->state = 2;
        s->finished_unreported.push_back(id);
    }
    s->active.swap(still);
    const long long budget = s->n_sm;
    if ((int)s->queued.size() >= kGroupMin) {
        // backlog: every queued request that gets a slot and arena room starts in one launch
        std::vector<ServeReq*> g;
        while (!s->queued.empty() && (int)s->active.size() < s->max_active) {
            ServeReq* q = s->reqs[s->queued.front()];
            size_t off = 0;
            if (!s->alloc->alloc(q->block_bytes, &off)) break;
            q->block_off = off;
            s->queued.pop_front();
            s->active.push_back(q->id);
            g.push_back(q);
        }
        if (!g.empty()) {
            const int rc = launch_group(s, g);
            if (rc > 0) {
                for (ServeReq* q : g) {  // no room for the group's block: one launch each
                    const int rc2 = launch_streamed(s, q);
                    if (rc2) return rc2;
                    s->inflight_sms += q->prep.R;
                }
            } else if (rc) {
                return rc;
            }
        }
    } else {
        while (!s->queued.empty() && (int)s->active.size() < s->max_active) {
            ServeReq* q = s->reqs[s->queued.front()];
            if (!s->active.empty() && s->inflight_sms + q->prep.R > budget) break;
            size_t off = 0;
            if (!s->alloc->alloc(q->block_bytes, &off)) break;
            q->block_off = off;
            s->queued.pop_front();
            const int rc = launch_streamed(s, q);
            if (rc) return rc;
            s->active.push_back(q->id);
            s->inflight_sms += q->prep.R;
        }
    }
    s->steps += 1;
    return PT_OK;
}

extern "C" int pt_server_step(pt_server* s, int64_t* done_ids, int32_t max_done, int32_t* n_done) {
    if (!s || !n_done || (max_done > 0 && !done_ids)) return PT_EINVAL;
    if (s->err) return s->err;
    if (s->streamed) {
        const int rc = step_streamed(s);
        if (rc) return rc;
        int n = 0;
        while (n < max_done && !s->finished_unreported.empty()) {
            done_ids[n++] = s->finished_unreported.front();
            s->finished_unreported.pop_front();
        }
        *n_done = n;
        return PT_OK;
    }
    int rc = admit(s);
    if (rc) return rc;
    if (!s->active.empty()) {
        std::vector<BatchInstance> insts;
        std::vector<int64_t> chunk(s->active.size());
        insts.reserve(s->active.size());
        for (size_t a = 0; a < s->active.size(); ++a) {
            ServeReq* q = s->reqs[s->active[a]];
            const int sps = q->inst.sweeps_per_swap;
            long long c = std::min<long long>(q->remaining, s->quantum);
            if (sps > 0 && c < q->remaining) c = std::max<long long>(sps, (c / sps) * sps);
            c = std::min<long long>(c, q->remaining);
            chunk[a] = c;
            BatchInstance I = q->inst;
            I.n_sweeps = (int)c;
            insts.push_back(I);
        }
        // ---- wide shape: every chain of every admitted request on its own CTA
        bool ran = false;
        if (s->wide) {
            std::vector<MultiProblem> mps(insts.size());
            std::vector<int2> wmap;
            size_t wsmem = 0;
            for (size_t a = 0; a < insts.size(); ++a) {
                const BatchInstance& I = insts[a];
                ServeReq* q = s->reqs[s->active[a]];
                MultiProblem& mp = mps[a];
                memset(&mp, 0, sizeof(mp));
                DevProblem& p = mp.p;
                p.desc = I.sdesc;
                p.items = I.items;
                p.level_off = I.level_off;
                p.thr = I.thr;
                p.coef = I.coef;
                p.spins = I.spins;
                p.E = I.E;
                p.M = I.M;
                p.rung_of_slot = I.rung_of_slot;
                p.slot_of_rung = I.slot_of_rung;
                p.acc = I.acc;
                p.swap_stats = I.swap_stats;
                p.mbox = (Mailbox*)(s->arena + q->block_off + q->prep.off_mbox);
                p.status = s->d_status;
                p.N = I.N;
                p.P = I.P;
                p.R = I.R;
                p.Lmax = I.Lmax;
                p.nL3 = I.nL3;
                p.n_levels = I.n_levels;
                p.dmax = I.dc;
                p.slot_stride = I.slot_stride;
                p.withhold_rung = -1;
                p.key0 = I.key0;
                p.key1 = I.key1;
                p.acc_in_smem = (size_t)I.R * kAccCount * 8 <= 16384 ? 1 : 0;
                p.tables_in_smem = (size_t)I.R * I.nL3 * 4 <= 49152 ? 1 : 0;
                if (p.tables_in_smem && multi_smem_bytes(p, I.dc) > s->smem_cap) p.tables_in_smem = 0;
                mp.dc = I.dc;
                mp.n_sweeps = I.n_sweeps;
                mp.sweeps_per_swap = I.sweeps_per_swap;
                mp.t0 = I.t0;
                mp.q0 = I.q0;
                mp.timeout_ns = 5000000000ll;
                wsmem = std::max(wsmem, multi_smem_bytes(p, I.dc));
                for (int rho = 0; rho < I.R; ++rho) wmap.push_back(make_int2((int)a, rho));
            }
            int per_sm = 0;
            const bool fits = wsmem <= s->smem_cap && (int)wmap.size() <= s->wmap_capacity &&
                              multi_prepare(s->wide_threads, wsmem, &per_sm) == cudaSuccess &&
                              (long long)per_sm * s->n_sm >= (long long)wmap.size();
            if (fits) {
                cudaError_t e;
                if ((e = cudaMemcpyAsync(s->d_multi, mps.data(), mps.size() * sizeof(MultiProblem),
                                         cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(s->d_wmap, wmap.data(), wmap.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                         s->stream)) != cudaSuccess ||
                    (e = launch_multi(s->d_multi, s->d_wmap, (int)wmap.size(), s->wide_threads, wsmem, s->stream)) !=
                        cudaSuccess)
                    return sfail(s, PT_ECUDA, "wide launch: %s", cudaGetErrorString(e));
                s->launches += 1;
                s->wide_steps += 1;
                ran = true;
            }
        }
        std::vector<int32_t> order(insts.size());
        for (size_t a = 0; a < order.size(); ++a) order[a] = (int32_t)a;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const double wx = (double)insts[x].N * insts[x].P * insts[x].R * (double)insts[x].n_sweeps;
            const double wy = (double)insts[y].N * insts[y].P * insts[y].R * (double)insts[y].n_sweeps;
            return wx > wy;
        });
        size_t smem = 0;
        for (const BatchInstance& I : insts) smem = std::max(smem, batch_smem_bytes(I, s->cluster, s->threads));
        cudaError_t e;
        if ((e = cudaMemcpyAsync(s->d_inst, insts.data(), insts.size() * sizeof(BatchInstance),
                                 cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->d_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 s->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(s->d_counter, 0, sizeof(int), s->stream)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        BatchParams bp;
        bp.inst = s->d_inst;
        bp.order = s->d_order;
        bp.count = (int)insts.size();
        bp.next_job = s->d_counter;
        bp.status = s->d_status;
        const int ncl = std::min<int>(s->n_clusters, (int)insts.size());
        if (!ran) {
            if ((e = launch_batch(bp, s->cluster, ncl, s->threads, smem, s->stream)) != cudaSuccess)
                return sfail(s, PT_ECUDA, "batch launch: %s", cudaGetErrorString(e));
            s->launches += 1;
        }
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
        {
            int st = 0;
            if ((e = cudaMemcpy(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
            if (st == PT_ETIMEDOUT) return sfail(s, PT_ETIMEDOUT, "a swap wait timed out");
            if (st) return sfail(s, PT_ECUDA, "device status %d", st);
        }
        s->steps += 1;
        std::vector<int64_t> still;
        for (size_t a = 0; a < s->active.size(); ++a) {
            ServeReq* q = s->reqs[s->active[a]];
            q->remaining -= chunk[a];
            q->inst.t0 += chunk[a];
            if (q->inst.sweeps_per_swap > 0) q->inst.q0 += chunk[a] / q->inst.sweeps_per_swap;
            if (q->remaining == 0) {
                q->state = 2;
                s->finished_unreported.push_back(q->id);
            } else {
                still.push_back(q->id);
            }
        }
        s->active.swap(still);
    }
    int n = 0;
    while (n < max_done && !s->finished_unreported.empty()) {
        done_ids[n++] = s->finished_unreported.front();
        s->finished_unreported.pop_front();
    }
    *n_done = n;
    return PT_OK;
}

extern "C" int pt_server_read_result(pt_server* s, int64_t id, int8_t* state, size_t bytes, pt_observables* o) {
    if (!s) return PT_EINVAL;
    if (s->err) return s->err;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, PT_EINVAL, "unknown request %lld", (long long)id);
    ServeReq* q = it->second;
    if (q->state != 2) return sfail(s, PT_EBUSY, "request %lld has not finished", (long long)id);
    const BatchInstance& I = q->inst;
    const int R = I.R;
    std::vector<int32_t> slot_of(R);
    std::vector<long long> E(R), M(R);
    std::vector<unsigned long long> acc((size_t)R * kAccCount), sw(2 * (size_t)R);
    std::vector<int8_t> spins;
    cudaError_t e;
    cudaStream_t st = s->stream;
    if ((e = cudaMemcpyAsync(slot_of.data(), I.slot_of_rung, R * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(E.data(), I.E, R * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(M.data(), I.M, R * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(acc.data(), I.acc, acc.size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sw.data(), I.swap_stats, sw.size() * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    if (state) {
        const size_t need = (size_t)R * I.N * I.P;
        if (bytes < need) return sfail(s, PT_EINVAL, "state buffer needs %zu bytes", need);
        spins.resize((size_t)R * I.slot_stride);
        if ((e = cudaMemcpyAsync(spins.data(), I.spins, spins.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return sfail(s, PT_ECUDA, "%s", cudaGetErrorString(e));
    if (state) {
        // replica order on the device, rung order across the boundary
        const size_t chain = (size_t)I.N * I.P;
        for (int r = 0; r < R; ++r) memcpy(state + (size_t)r * chain, &spins[(size_t)slot_of[r] * I.slot_stride], chain);
    }
    if (o) {
        o->t = I.t0;
        o->q = I.q0;
        for (int r = 0; r < R; ++r) {
            const int slot = slot_of[r];
            if (o->E) o->E[r] = E[slot];
            if (o->M) o->M[r] = M[slot];
            const unsigned long long* a = &acc[(size_t)r * kAccCount];
            if (o->n_meas) o->n_meas[r] = (int64_t)a[kAccN];
            if (o->sum_E) o->sum_E[r] = (int64_t)a[kAccE];
            if (o->sum_E2) o->sum_E2[r] = (int64_t)a[kAccE2];
            if (o->sum_M) o->sum_M[r] = (int64_t)a[kAccM];
            if (o->sum_M2) o->sum_M2[r] = (int64_t)a[kAccM2];
            if (o->flip_acc) o->flip_acc[r] = (int64_t)a[kAccFlip];
            if (o->replica_at) o->replica_at[r] = slot;
        }
        for (int r = 0; r + 1 < R; ++r) {
            if (o->swap_att) o->swap_att[r] = (int64_t)sw[2 * r];
            if (o->swap_acc) o->swap_acc[r] = (int64_t)sw[2 * r + 1];
        }
    }
    return PT_OK;
}

extern "C" int pt_server_release(pt_server* s, int64_t id) {
    if (!s) return PT_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, PT_EINVAL, "unknown request %lld", (long long)id);
    ServeReq* q = it->second;
    if (q->state == 1) return sfail(s, PT_EBUSY, "request %lld is still running", (long long)id);
    if (q->state == 0) s->queued.erase(std::find(s->queued.begin(), s->queued.end(), id));
    if (q->state == 2) s->alloc->release(q->block_off, q->block_bytes);
    if (q->done) cudaEventDestroy(q->done);
    delete q;
    s->reqs.erase(it);
    return PT_OK;
}

extern "C" int pt_server_get_info(const pt_server* s, pt_server_info* o) {
    if (!s || !o) return PT_EINVAL;
    o->active = (int32_t)s->active.size();
    o->queued = (int32_t)s->queued.size();
    o->arena_bytes = (int64_t)s->alloc->size();
    o->arena_used = (int64_t)s->alloc->used();
    o->steps = s->steps;
    o->kernel_launches = s->launches;
    o->wide_steps = s->wide_steps;
    o->group_launches = s->group_launches;
    return PT_OK;
}

extern "C" int pt_server_destroy(pt_server* s) {
    if (!s) return PT_OK;
    cudaStreamSynchronize(s->stream);
    free_server(s);
    return PT_OK;
}

extern "C" const char* pt_server_last_error(const pt_server* s) { return s ? s->msg : g_srv_create_msg; }
