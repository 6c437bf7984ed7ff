// sched.cuh -- device-side task scheduler of the tiled QR (Sec. 4): the task
// graph of Algorithm 2 executed by one persistent kernel.  Each task has a
// dependency counter; the task that completes a counter pushes the successor
// onto one of four ready queues, one per priority level of Sec. 4 (DGEQRT >
// DTSQRT > DLARFB > DSSRFB).  Workers (one CTA each) pop the highest-priority
// ready task.  Queues are write-once arrays sized to the exact number of tasks
// of their kind, so a slot is never reused and a pop only advances the head
// (a CAS, or on the bulk level an atomicAdd, see q_try_pop).
//
// Progress does not depend on CTA co-residency: a CTA only ever waits while
// idle (never while holding a task), and every wait is bounded by a
// watchdog that records TILEQR_ERR_TIMEOUT and returns.
#pragma once
#include "common.cuh"

namespace tqr {

struct Queues {
    SchedCtrl *ctrl;
    unsigned int *cnt;
    unsigned long long *slot[K_NKIND];
    unsigned int cap[K_NKIND];
    unsigned int total;
    unsigned long long watchdog_ns;
    unsigned long long withheld;   // task code never released (watchdog test), ~0 = none
    unsigned long long *trace;     // optional per-task trace records (4 u64 each)
    unsigned int trace_cap;
    // stress test of the schedule: nonzero = a seed; every task then sleeps
    // a pseudo-random time (up to ~40 us) before it runs and before it
    // releases its successors, so tasks finish in orders the natural timing
    // rarely gives.  0 (the default) = off.
    unsigned long long delay_seed = 0;
};

// The stress-test delay of a task, in ns (a SplitMix64-style mix of the
// task code, the seed and the site).
__device__ __forceinline__ unsigned int stress_delay_ns(unsigned long long code, unsigned long long seed, int site)
{
    unsigned long long z = code * 0x9E3779B97F4A7C15ull + seed + (unsigned long long)site * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (unsigned int)(z % 20000u);
}
__device__ __forceinline__ void stress_sleep(unsigned int ns)
{
    __nanosleep(ns);
    __nanosleep(ns);
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void q_push(const Queues &Q, int level, unsigned long long code)
{
    if (code == Q.withheld)
        return;
    const unsigned int s = atomicAdd(&Q.ctrl->tail[level], 1u);
    if (s < Q.cap[level])
        st_release_u64(&Q.slot[level][s], code + 1ull);
    else
        atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_CUDA);  // cannot happen: capacities are exact
}

// The last level holds the bulk of every graph (the DSSRFB-class updates),
// and with short tasks (the tensor-core updates run in tens of microseconds)
// the CTAs pop it several times per microsecond.  A compare-and-swap on its
// head then fails and retries under contention, so while that level has more
// than TICKET_MARGIN tasks queued a CTA claims the next slot with one
// atomicAdd instead.  A claimed slot that has not been filled yet (the head
// ran past the tail between the loads and the add) stays the CTA's "ticket":
// its task will be this CTA's next bulk task, and until it is pushed the CTA
// keeps popping the higher levels.  Every slot below the head is owned by
// some CTA that runs its task once it is filled, so no ready task is ever
// stranded; a ticket at or beyond the capacity claims nothing.
constexpr int Q_BULK = K_NKIND - 1;
constexpr unsigned int NO_TICKET = 0xFFFFFFFFu;
constexpr unsigned int TICKET_MARGIN = 8;

__device__ __forceinline__ bool q_try_pop(const Queues &Q, unsigned long long &code, unsigned int &ticket)
{
    unsigned int hd[K_NKIND], tl[K_NKIND];
#pragma unroll
    for (int l = 0; l < K_NKIND; l++) {
        hd[l] = ld_relaxed_u32(&Q.ctrl->head[l]);
        tl[l] = ld_relaxed_u32(&Q.ctrl->tail[l]);
    }
    for (int lvl = 0; lvl < K_NKIND; lvl++) {
        if (lvl == Q_BULK && ticket != NO_TICKET) {
            const unsigned long long v = ld_acquire_u64(&Q.slot[lvl][ticket]);
            if (v == 0ull)
                return false;
            code = v - 1ull;
            ticket = NO_TICKET;
            return true;
        }
        if (hd[lvl] >= Q.cap[lvl] || hd[lvl] >= tl[lvl])
            continue;   // empty as of the loads
        if (lvl == Q_BULK && tl[lvl] - hd[lvl] > TICKET_MARGIN) {
            const unsigned int t = atomicAdd(&Q.ctrl->head[lvl], 1u);
            if (t >= Q.cap[lvl])
                return false;
            // the slot is this CTA's; its push may still be in flight
            for (int spin = 0; spin < 4; spin++) {
                const unsigned long long v = ld_acquire_u64(&Q.slot[lvl][t]);
                if (v != 0ull) {
                    code = v - 1ull;
                    return true;
                }
            }
            ticket = t;
            return false;
        }
        for (;;) {
            const unsigned int h = ld_relaxed_u32(&Q.ctrl->head[lvl]);
            if (h >= Q.cap[lvl])
                break;
            const unsigned long long v = ld_acquire_u64(&Q.slot[lvl][h]);
            if (v == 0ull)
                break;  // empty, or a push still in flight
            if (atomicCAS(&Q.ctrl->head[lvl], h, h + 1u) == h) {
                code = v - 1ull;
                return true;
            }
        }
    }
    return false;
}

enum { CMD_RUN = 1, CMD_EXIT = 2 };

// Thread 0 of a worker CTA: wait (bounded) for a ready task.  `ticket` is
// the CTA's claim on a bulk-level slot (NO_TICKET: none), kept by the caller
// across calls.
__device__ __noinline__ static int q_acquire(const Queues &Q, unsigned long long &code, unsigned int &ticket)
{
    unsigned long long t_last = globaltimer_ns();
    unsigned int last_done = ld_relaxed_u32(&Q.ctrl->completed);
    unsigned int backoff = 32;
    const unsigned long long max_iter = 1ull << 27;
    for (unsigned long long it = 0; it < max_iter; it++) {
        if (ld_relaxed_s32(&Q.ctrl->error) != 0)
            return CMD_EXIT;
        if (q_try_pop(Q, code, ticket)) {
            __threadfence();
            return CMD_RUN;
        }
        const unsigned int done = ld_relaxed_u32(&Q.ctrl->completed);
        if (done >= Q.total)
            return CMD_EXIT;
        const unsigned long long now = globaltimer_ns();
        if (done != last_done) {
            last_done = done;
            t_last = now;
        } else if (now - t_last > Q.watchdog_ns) {
            atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_TIMEOUT);
            return CMD_EXIT;
        }
        __nanosleep(backoff);
        backoff = backoff < 1024 ? backoff * 2 : 1024;
    }
    atomicCAS(&Q.ctrl->error, 0, TILEQR_ERR_TIMEOUT);
    return CMD_EXIT;
}

// Signal one successor: the call that completes its counter releases it.
__device__ __forceinline__ void q_signal(const Queues &Q, size_t cnt_idx, int ndeps, int level,
                                         unsigned long long code)
{
    __threadfence();
    const unsigned int old = atomicAdd(&Q.cnt[cnt_idx], 1u);
    if ((int)old + 1 == ndeps) {
        __threadfence();
        q_push(Q, level, code);
    }
}

__device__ __forceinline__ void trace_record(const Queues &Q, unsigned long long code,
                                             unsigned long long t0, unsigned long long t1)
{
    if (Q.trace == nullptr)
        return;
    const unsigned int s = atomicAdd(&Q.ctrl->trace_cursor, 1u);
    if (s < Q.trace_cap) {
        unsigned int smid;
        asm volatile("mov.u32 %0, %smid;" : "=r"(smid));
        unsigned long long *rec = Q.trace + 4ull * s;
        rec[0] = code;
        rec[1] = t0;
        rec[2] = t1;
        rec[3] = smid;
    }
}

}  // namespace tqr
