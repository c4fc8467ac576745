// pt_noalloc.cu -- pt_run_noalloc: the byte-wise sweep kernel with in-launch swaps, run on
// device buffers the caller owns, with no allocation of any kind.
//
// Who needs this: callers that cannot allocate device memory, neither themselves nor
// through this library. Latency-critical loops must not enter the allocator (cudaMalloc
// and cudaFree can synchronise the device and take locks shared with other threads);
// embedding runtimes and frameworks often hand out device memory only from their own pool
// and account for every byte; and some deployments fix the process's device memory at
// start-up. pt_create allocates, so such callers prepare the problem with the host-only
// helpers, copy it into memory they own, and call this.
//
// The one piece of scratch memory the kernel needs, the swap mailboxes, is the file-scope
// array below: PT_NOALLOC_MAILBOXES entries of 16 bytes (256 KiB), which every GPU that
// loads this library keeps until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "pt.h"
#include "pt_internal.h"

using namespace ptq;

static_assert(sizeof(Mailbox) == 16, "mailbox entries are 16 bytes");

static __device__ __align__(256) Mailbox g_noalloc_mailboxes[PT_NOALLOC_MAILBOXES];

// In host code `g_noalloc_mailboxes` only names a host-side stand-in for the symbol; the
// device address is looked up once per device (with that device current) and cached here.
// A device reset (cudaDeviceReset) makes a cached address stale, so the entry point must not
// be called on a device after its reset.
static std::mutex g_setup_lock;
static void* g_mailbox_addr[256];
static bool g_mailbox_ready[256];

static thread_local char g_noalloc_msg[256] = "";

static int fail(int code, const char* msg) {
    strncpy(g_noalloc_msg, msg, sizeof(g_noalloc_msg) - 1);
    g_noalloc_msg[sizeof(g_noalloc_msg) - 1] = 0;
    return code;
}

extern "C" const char* pt_noalloc_last_error(void) { return g_noalloc_msg; }

static int mailbox_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return fail(PT_ENODEV, "no current CUDA device");
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_mailbox_ready[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_mailboxes);
        if (e != cudaSuccess || ptr == nullptr) return fail(PT_ECUDA, "cudaGetSymbolAddress of the mailbox array failed");
        g_mailbox_addr[dev] = ptr;
        g_mailbox_ready[dev] = true;
    }
    *out = g_mailbox_addr[dev];
    return PT_OK;
}

extern "C" int pt_run_noalloc(const pt_device_problem* q, int64_t n_sweeps, int32_t sweeps_per_swap,
                              int32_t wait_timeout_ms, void* cuda_stream) {
    if (!q) return fail(PT_EINVAL, "null problem");
    if (q->n < 1 || q->n > 65535 || (q->P != 1 && (q->P < 2 || (q->P & 1) || q->P > 4096)) || q->R < 1 || q->R > 65535)
        return fail(PT_EINVAL, "need 1 <= n <= 65535, even 2 <= P <= 4096, 1 <= R <= 65535");
    if (q->lmax < 0 || q->lmax > 127) return fail(PT_EINVAL, "lmax must be in [0, 127]");
    if (q->row_stride != 4 && q->row_stride != 8 && q->row_stride != 32)
        return fail(PT_EINVAL, "row_stride must be 4, 8 or 32");
    if (q->n_levels < 1 || q->n_levels > 2 * q->n) return fail(PT_EINVAL, "n_levels out of range");
    if (!q->nbr || !q->h || !q->items || !q->level_off || !q->thr || !q->coef || !q->spins || !q->E || !q->M ||
        !q->rung_of_slot || !q->slot_of_rung || !q->stats || !q->swap_stats || !q->status)
        return fail(PT_EINVAL, "a device pointer is null");
    if (((uintptr_t)q->spins & 15) != 0) return fail(PT_EINVAL, "spins must be 16-byte aligned");
    if (n_sweeps < 0 || sweeps_per_swap < 0 || sweeps_per_swap > (1 << 30))
        return fail(PT_EINVAL, "need n_sweeps >= 0 and 0 <= sweeps_per_swap <= 2^30");
    if (q->t0 < 0 || q->q0 < 0 || q->t0 + n_sweeps > 0xFFFFFFFFll ||
        (sweeps_per_swap > 0 && q->q0 + n_sweeps / sweeps_per_swap > 0xFFFFFFFFll))
        return fail(PT_EOVERFLOW, "sweep or swap-pass counter would exceed 2^32 - 1");
    const bool swaps = sweeps_per_swap > 0 && q->R > 1;
    if (swaps && q->R > PT_NOALLOC_MAILBOXES)
        return fail(PT_EINVAL, "more rungs than the fixed mailbox array holds (PT_NOALLOC_MAILBOXES)");

    void* mbox = nullptr;
    int rc = mailbox_address(&mbox);
    if (rc) return rc;

    DevProblem p;
    memset(&p, 0, sizeof(p));
    p.nbr = q->nbr;
    p.h = q->h;
    p.items = q->items;
    p.level_off = q->level_off;
    p.thr = q->thr;
    p.coef = q->coef;
    p.spins = q->spins;
    p.E = (long long*)q->E;
    p.M = (long long*)q->M;
    p.rung_of_slot = q->rung_of_slot;
    p.slot_of_rung = q->slot_of_rung;
    p.acc = (unsigned long long*)q->stats;
    p.swap_stats = (unsigned long long*)q->swap_stats;
    p.mbox = (Mailbox*)mbox;
    p.status = q->status;
    p.N = q->n;
    p.P = q->P;
    p.R = q->R;
    p.Lmax = q->lmax;
    p.nL3 = (2 * q->lmax + 1) * 3;
    p.n_levels = q->n_levels;
    p.dmax = q->row_stride;
    p.slot_stride = (int)(((size_t)q->n * q->P + 15) & ~(size_t)15);
    p.withhold_rung = -1;
    p.key0 = (uint32_t)(q->seed & 0xFFFFFFFFu);
    p.key1 = (uint32_t)(q->seed >> 32);

    int dev = 0, max_smem = 0, n_sm = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    p.acc_in_smem = (size_t)q->R * kAccCount * 8 <= 16384 ? 1 : 0;
    p.tables_in_smem = (size_t)q->R * p.nL3 * 4 <= 49152 ? 1 : 0;
    LaunchPlan plan;
    plan.path = kPathGeneric;
    plan.dclass = q->row_stride;
    if (p.tables_in_smem && sweep_smem_bytes(p, kPathGeneric, plan.dclass) > (size_t)max_smem) p.tables_in_smem = 0;
    if (p.acc_in_smem && sweep_smem_bytes(p, kPathGeneric, plan.dclass) > (size_t)max_smem) p.acc_in_smem = 0;
    plan.smem_bytes = sweep_smem_bytes(p, kPathGeneric, plan.dclass);
    if (plan.smem_bytes > (size_t)max_smem) return fail(PT_EINVAL, "one chain does not fit in shared memory");
    {
        int G = ((q->P / 2) + 3) / 4, Gp = 1;
        while (Gp < G) Gp <<= 1;
        const long long units = 2ll * q->n * Gp;
        long long avg = (units + q->n_levels - 1) / q->n_levels;
        avg = ((avg + 31) / 32) * 32;
        plan.threads = (int)(avg < 128 ? 128 : (avg > 512 ? 512 : avg));
    }
    plan.n_consumer = plan.threads;
    if (prepare_sweep_kernel(plan) != cudaSuccess) return fail(PT_ECUDA, "cudaFuncSetAttribute failed");
    if (swaps) {
        int per_sm = 0;
        if (sweep_kernel_occupancy(p, plan, &per_sm) != cudaSuccess || !coop || (long long)per_sm * n_sm < q->R)
            return fail(PT_EINVAL, "all chains must be resident at once for swaps inside the launch");
    }

    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long timeout_ns = (long long)(wait_timeout_ms > 0 ? wait_timeout_ms : 5000) * 1000000ll;
    const long long max_passes = swaps ? (long long)(PT_NOALLOC_MAILBOXES / q->R) : 0;
    long long t = q->t0, qq = q->q0, done = 0;
    const long long full = swaps ? (n_sweeps / sweeps_per_swap) * sweeps_per_swap : 0;
    while (done < n_sweeps) {
        long long chunk, passes = 0;
        int sps = 0;
        if (done < full) {
            // whole swap intervals only, so that every launch starts on an interval boundary
            // and the passes fall on the same sweeps as in one long run
            chunk = full - done;
            if (chunk > max_passes * sweeps_per_swap) chunk = max_passes * sweeps_per_swap;
            const long long cap = ((1ll << 30) / sweeps_per_swap) * sweeps_per_swap;
            if (chunk > cap) chunk = cap;
            passes = chunk / sweeps_per_swap;
            sps = sweeps_per_swap;
            // every call shares the array; a mailbox left by an earlier call could carry a
            // matching tag, so the entries this launch reads start at zero
            if (cudaMemsetAsync(mbox, 0, (size_t)passes * q->R * sizeof(Mailbox), s) != cudaSuccess)
                return fail(PT_ECUDA, "clearing the mailboxes failed");
        } else {
            chunk = n_sweeps - done;
            if (chunk > (1ll << 30)) chunk = 1ll << 30;
        }
        if (launch_sweeps(p, plan, t, qq, (int)chunk, sps, timeout_ns, sps > 0, s) != cudaSuccess)
            return fail(PT_ECUDA, "sweep launch failed");
        t += chunk;
        qq += passes;
        done += chunk;
    }
    return PT_OK;
}
