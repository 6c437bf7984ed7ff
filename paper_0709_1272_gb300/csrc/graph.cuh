// graph.cuh -- the task graph of the tiled QR with an elimination tree, as
// host/device functions: task kinds, dependency counts and successor lists.
//
// Algorithm 2 eliminates the tiles of panel column k by one DTSQRT chain
// into the diagonal tile (a flat tree).  The tree form splits the rows
// k..p-1 of step k into domains of H consecutive tile rows starting at row
// k: the head of each domain is reduced by DGEQRT (and its row updated by
// DLARFB), the other rows of the domain are eliminated into the head by the
// DTSQRT / DSSRFB chain of Algorithm 2, and the domain heads are then merged
// pairwise by the triangle-on-triangle kernels DTTQRT / DTTMQR: at level l,
// the head of domain d + 2^l into the head of domain d, d a multiple of
// 2^(l+1).  The chain length per step drops from p - k to H + ceil(log2 of
// the domain count).  H >= p - k leaves one domain: exactly Algorithm 2.
//
// A task is (tt, k, i, j): step k, tile row i, tile column j; tt = 1 marks the
// tree kernels (DTTQRT at j == k, DTTMQR at j > k, both on domain head i).
// For tt = 0 the kind follows from j == k and whether row i heads a domain.
// Dependencies (from the tiles each kernel reads and writes):
//   GEQRT(i,k)   <- previous-step writer of tile (i,k)
//   TSQRT(i,k)   <- GEQRT / TSQRT of the row above in the domain; prev. step
//   TTQRT(e,k)   <- last writer of head e's R; last writer of the partner's R
//   LARFB(i,j,k) <- GEQRT(i,k); prev. step
//   SSRFB(i,j,k) <- TSQRT(i,k); last update of the head's tile (head, j); prev.
//   TTMQR(e,j,k) <- TTQRT(e,k); last update of tile (e,j); of (partner, j)
// The last writer of a tile at step k releases the first task of step k+1 on
// it.  Every task is released by exactly ndeps signals.
#pragma once
#include "common.cuh"

namespace tqr {

enum { K_TTQRT = 4, K_TTMQR = 5 };

// Ready-queue level of a task (the four priorities of Sec. 4; the tree's
// merge joins the panel level, its update the row-update level).  An update
// of column k+1 (j == k + 1) feeds the next step's panel, so it moves up one
// level: otherwise it waits behind the whole backlog of its kind and delays
// every later step.
__host__ __device__ inline int kind_prio(int kind, int k = -1, int j = -2)
{
    const int base = kind < 4 ? kind : (kind == K_TTQRT ? 1 : 2);
    const bool update = kind == K_LARFB || kind == K_SSRFB || kind == K_TTMQR;
    return (update && j == k + 1) ? base - 1 : base;
}

struct TGraph {
    int p, q, steps, H;   // 1 <= H <= p
};

__host__ __device__ inline TGraph make_graph(int p, int q, int h)
{
    TGraph G;
    G.p = p;
    G.q = q;
    G.steps = p < q ? p : q;
    G.H = (h <= 0 || h > p) ? (p > 0 ? p : 1) : h;
    return G;
}

__host__ __device__ inline int g_ctz(int d)
{
    int l = 0;
    while (!((d >> l) & 1))
        l++;
    return l;
}
__host__ __device__ inline int g_ndom(const TGraph &G, int k) { return (G.p - k + G.H - 1) / G.H; }
__host__ __device__ inline int g_head(const TGraph &G, int k, int d) { return k + d * G.H; }
__host__ __device__ inline int g_dom(const TGraph &G, int k, int i) { return (i - k) / G.H; }
__host__ __device__ inline int g_last(const TGraph &G, int k, int d)
{
    const int e = k + (d + 1) * G.H;
    return (e < G.p ? e : G.p) - 1;
}
// Number of merges into domain d at step k (levels 0 .. L-1 exist).
__host__ __device__ inline int g_nmerge(const TGraph &G, int k, int d)
{
    const int nd = g_ndom(G, k);
    const int lim = d == 0 ? 30 : g_ctz(d);
    int n = 0;
    while (n < lim && d + (1 << n) < nd)
        n++;
    return n;
}
// Partner (merge target) row of domain head e at step k.
__host__ __device__ inline int g_partner(const TGraph &G, int k, int e)
{
    const int d = g_dom(G, k, e);
    return g_head(G, k, d - (1 << g_ctz(d)));
}

__host__ __device__ inline int g_kind(const TGraph &G, int tt, int k, int i, int j)
{
    if (tt)
        return j == k ? K_TTQRT : K_TTMQR;
    const bool head = ((i - k) % G.H) == 0;
    if (j == k)
        return head ? K_GEQRT : K_TSQRT;
    return head ? K_LARFB : K_SSRFB;
}

__host__ __device__ inline int g_ndeps(int kind, int k)
{
    const int prev = k > 0 ? 1 : 0;
    switch (kind) {
    case K_GEQRT: return prev;
    case K_TSQRT: return 1 + prev;
    case K_LARFB: return 1 + prev;
    case K_SSRFB: return 2 + prev;
    case K_TTQRT: return 2;
    default: return 3;
    }
}

struct GTask {
    int tt, k, i, j;
};

// Dependency counter index of a task (tt = 1 tasks follow all tt = 0 ones).
__host__ __device__ inline size_t g_cidx(const TGraph &G, int tt, int k, int i, int j)
{
    return (((size_t)tt * G.steps + k) * G.p + i) * G.q + j;
}
__host__ __device__ inline size_t g_ncounters(const TGraph &G)
{
    return (size_t)(G.H < G.p ? 2 : 1) * G.steps * G.p * G.q;
}

// The task that next writes head(d)'s tile in column j after the level-lev
// merge into domain d (lev = -1: after d's own chain), if any: the level
// lev+1 merge into d, else d's own merge into its partner (d > 0).
__host__ __device__ inline int g_next_merge(const TGraph &G, int k, int d, int lev, int j, GTask *out)
{
    if (lev + 1 < g_nmerge(G, k, d)) {
        *out = GTask{1, k, g_head(G, k, d + (1 << (lev + 1))), j};
        return 1;
    }
    if (d > 0) {
        *out = GTask{1, k, g_head(G, k, d), j};
        return 1;
    }
    return 0;
}

// Successors: a fan-out over the columns right of the panel (factor kinds:
// their row of updates), then up to two specific tasks.
__host__ __device__ inline int g_fanout(const TGraph &G, int kind, int k)
{
    return (kind == K_GEQRT || kind == K_TSQRT || kind == K_TTQRT) ? G.q - k - 1 : 0;
}
__host__ __device__ inline GTask g_fan_task(int kind, int k, int i, int s)
{
    return GTask{kind == K_TTQRT ? 1 : 0, k, i, k + 1 + s};
}
__host__ __device__ inline int g_specific(const TGraph &G, int kind, int k, int i, int j, GTask out[2])
{
    int n = 0;
    switch (kind) {
    case K_GEQRT:
    case K_LARFB:
    case K_TSQRT: {
        // next in the domain's chain, else the first merge that needs it
        const int d = g_dom(G, k, i);
        if (g_last(G, k, d) > i)
            out[n++] = GTask{0, k, i + 1, j};
        else
            n += g_next_merge(G, k, d, -1, j, out + n);
        break;
    }
    case K_SSRFB: {
        const int d = g_dom(G, k, i);
        if (g_last(G, k, d) > i)
            out[n++] = GTask{0, k, i + 1, j};
        else
            n += g_next_merge(G, k, d, -1, j, out + n);
        if (k + 1 < G.steps)
            out[n++] = GTask{0, k + 1, i, j};
        break;
    }
    case K_TTQRT: {
        const int d = g_dom(G, k, i);
        n += g_next_merge(G, k, d - (1 << g_ctz(d)), g_ctz(d), j, out + n);
        break;
    }
    default: {   // K_TTMQR
        const int d = g_dom(G, k, i);
        n += g_next_merge(G, k, d - (1 << g_ctz(d)), g_ctz(d), j, out + n);
        if (k + 1 < G.steps)
            out[n++] = GTask{0, k + 1, i, j};
        break;
    }
    }
    return n;
}

// Tasks of each kind in the whole graph.
__host__ inline void g_count(const TGraph &G, unsigned long long cnt[6])
{
    for (int t = 0; t < 6; t++)
        cnt[t] = 0;
    for (int k = 0; k < G.steps; k++) {
        const unsigned long long P = G.p - k, nd = g_ndom(G, k), nq = G.q - k - 1;
        cnt[K_GEQRT] += nd;
        cnt[K_TSQRT] += P - nd;
        cnt[K_TTQRT] += nd - 1;
        cnt[K_LARFB] += nd * nq;
        cnt[K_SSRFB] += (P - nd) * nq;
        cnt[K_TTMQR] += (nd - 1) * nq;
    }
}

// ---------------------------------------------------------------------------
// Q^T applied to right-hand sides: per column chunk, the update kinds of the
// graph restricted to one tile column (tasks (tt, k, i); a row block of B
// plays the part of tile (i, j)): LB = DLARFB on a head row, SB = DSSRFB on
// a domain row, TB = DTTMQR merging two head rows.
__host__ __device__ inline int ga_kind(const TGraph &G, int tt, int k, int i)
{
    if (tt)
        return K_TTMQR;
    return ((i - k) % G.H) == 0 ? K_LARFB : K_SSRFB;
}
__host__ __device__ inline int ga_ndeps(int kind, int k)
{
    const int prev = k > 0 ? 1 : 0;
    return kind == K_LARFB ? prev : (kind == K_SSRFB ? 1 + prev : 2);
}
__host__ __device__ inline int ga_specific(const TGraph &G, int kind, int k, int i, GTask out[2])
{
    GTask t[2];
    int n = 0;
    if (kind == K_LARFB || kind == K_SSRFB) {
        const int d = g_dom(G, k, i);
        if (g_last(G, k, d) > i)
            t[n++] = GTask{0, k, i + 1, 0};
        else
            n += g_next_merge(G, k, d, -1, 0, t + n);
    } else {
        const int d = g_dom(G, k, i);
        n += g_next_merge(G, k, d - (1 << g_ctz(d)), g_ctz(d), 0, t + n);
    }
    if (kind != K_LARFB && k + 1 < G.steps)
        t[n++] = GTask{0, k + 1, i, 0};
    for (int s = 0; s < n; s++)
        out[s] = t[s];
    return n;
}
// Tasks per ready-queue level (kind_prio), for the write-once queues.
__host__ inline void g_level_counts(const TGraph &G, unsigned long long caps[K_NKIND])
{
    for (int t = 0; t < K_NKIND; t++)
        caps[t] = 0;
    for (int k = 0; k < G.steps; k++) {
        const unsigned long long P = G.p - k, nd = g_ndom(G, k), nq = G.q - k - 1;
        const unsigned long long c1 = nq > 0 ? 1 : 0, rest = nq > 0 ? nq - 1 : 0;
        caps[0] += nd;                              // GEQRT
        caps[1] += (P - nd) + (nd - 1);             // TSQRT, TTQRT
        caps[1] += nd * c1 + (nd - 1) * c1;         // LARFB, TTMQR on column k+1
        caps[2] += nd * rest + (nd - 1) * rest;     // the other LARFB, TTMQR
        caps[2] += (P - nd) * c1;                   // SSRFB on column k+1
        caps[3] += (P - nd) * rest;                 // the other SSRFB
    }
}

// Q itself (tileqr_apply_q) runs the same tasks in the reverse graph: a task
// is released by its forward successors (count: ga_specific) and on
// completion signals its forward predecessors, listed here:
//   LB(h,k)  <- last writer of row h at step k-1 (k > 0)
//   SB(r,k)  <- LB(head) or SB(r-1,k) (the domain chain); last writer of row r at k-1
//   TB(e,k)  <- last writer of head e's row before its merge (the level L(e)-1
//               merge into e, else e's chain end); the same for the partner d
//               before the level-l merge (level l-1 merge into d, else d's end)
// The last writer of row r at step k' is SB(r,k') if r is not a domain head
// there, else TB(r,k') (r > k').
__host__ __device__ inline GTask ga_last_writer(const TGraph &G, int k, int r)
{
    return ((r - k) % G.H) == 0 ? GTask{1, k, r, 0} : GTask{0, k, r, 0};
}
__host__ __device__ inline GTask ga_chain_end(const TGraph &G, int k, int d)
{
    return GTask{0, k, g_last(G, k, d), 0};   // SB(last) or, for a one-row domain, LB(head)
}
__host__ __device__ inline int ga_predecessors(const TGraph &G, int kind, int k, int i, GTask out[2])
{
    int n = 0;
    if (kind == K_LARFB) {
        if (k > 0)
            out[n++] = ga_last_writer(G, k - 1, i);
    } else if (kind == K_SSRFB) {
        out[n++] = GTask{0, k, i - 1, 0};
        if (k > 0)
            out[n++] = ga_last_writer(G, k - 1, i);
    } else {
        const int e = g_dom(G, k, i), lev = g_ctz(e), d = e - (1 << lev);
        const int le = g_nmerge(G, k, e);
        out[n++] = le > 0 ? GTask{1, k, g_head(G, k, e + (1 << (le - 1))), 0} : ga_chain_end(G, k, e);
        out[n++] = lev > 0 ? GTask{1, k, g_head(G, k, d + (1 << (lev - 1))), 0} : ga_chain_end(G, k, d);
    }
    return n;
}

__host__ inline void ga_count(const TGraph &G, unsigned long long cnt[2])
{
    cnt[0] = cnt[1] = 0;   // [0]: LB, [1]: SB + TB
    for (int k = 0; k < G.steps; k++) {
        cnt[0] += g_ndom(G, k);
        cnt[1] += (G.p - k) - 1;
    }
}

// ---------------------------------------------------------------------------
// The tiled Cholesky factorization (Sec. 3.1, Algorithm 1) on p x p tiles:
// tasks (k, i, j) with k <= j <= i: DPOTF2 (k,k,k), DTRSM (i,k,k), DGSMM
// (i,j,k), j > k.  Dependencies (from the tiles each kernel reads/writes):
//   DPOTF2(k)    <- DGSMM(k,k,k-1)
//   DTRSM(i,k)   <- DPOTF2(k); DGSMM(i,k,k-1)
//   DGSMM(i,j,k) <- DTRSM(i,k); DTRSM(j,k) (j < i); DGSMM(i,j,k-1)
// The DGSMMs of column k+1 feed the next step's panel and get the higher of
// the two update priority levels.
enum { KC_POTF2 = 0, KC_TRSM = 1, KC_GSMM = 2 };

__host__ __device__ inline int cg_kind(int k, int i, int j)
{
    return (j == k) ? (i == k ? KC_POTF2 : KC_TRSM) : KC_GSMM;
}
__host__ __device__ inline int cg_prio(int kind, int k, int j)
{
    return kind == KC_POTF2 ? 0 : (kind == KC_TRSM ? 1 : (j == k + 1 ? 2 : 3));
}
__host__ __device__ inline int cg_ndeps(int k, int i, int j)
{
    const int prev = k > 0 ? 1 : 0;
    switch (cg_kind(k, i, j)) {
    case KC_POTF2: return prev;
    case KC_TRSM: return 1 + prev;
    default: return (i == j ? 1 : 2) + prev;
    }
}
__host__ __device__ inline size_t cg_cidx(int p, int k, int i, int j)
{
    return ((size_t)k * p + i) * p + j;
}
// successors: DPOTF2(k) -> DTRSM(i,k), i > k;  DTRSM(i,k) -> DGSMM(i,j,k),
// k < j <= i, and DGSMM(i',i,k), i' > i;  DGSMM(i,j,k) -> the step-(k+1)
// task on tile (i,j)
__host__ __device__ inline int cg_nsucc(int p, int k, int i, int j)
{
    switch (cg_kind(k, i, j)) {
    case KC_POTF2: return p - k - 1;
    case KC_TRSM: return p - k - 1;
    default: return 1;
    }
}
__host__ __device__ inline GTask cg_succ(int p, int k, int i, int j, int s)
{
    switch (cg_kind(k, i, j)) {
    case KC_POTF2: return GTask{0, k, k + 1 + s, k};
    case KC_TRSM:
        if (s < i - k)
            return GTask{0, k, i, k + 1 + s};                  // row i: DGSMM(i, j, k)
        return GTask{0, k, i + 1 + (s - (i - k)), i};          // column i: DGSMM(i', i, k)
    default: return GTask{0, k + 1, i, j};
    }
}
__host__ inline void cg_count(int p, unsigned long long cnt[4])
{
    for (int t = 0; t < 4; t++)
        cnt[t] = 0;
    for (int k = 0; k < p; k++) {
        const unsigned long long r = p - k - 1;
        cnt[0] += 1;
        cnt[1] += r;
        cnt[2] += r;                          // DGSMM on column k+1
        cnt[3] += r * (r + 1) / 2 - r;        // the other DGSMMs
    }
}


// ---------------------------------------------------------------------------
// The tiled LU with tiled pairwise pivoting (Sec. 3.2.2, Algorithm 3) has the
// task graph of Algorithm 2 (the flat tree) kernel for kernel: DGETRF reads
// and writes the diagonal tile like DGEQRT, DGESSM reads its multipliers
// like DLARFB, DTSTRF chains on U_kk like DTSQRT on R_kk, and DSSSSM updates
// the pair (U_kj, A_ij) like DSSRFB.  The LU path therefore runs the graph
// functions above with H = p; these are the LU names of the four kinds.
enum { KL_GETRF = 0, KL_GESSM = 1, KL_TSTRF = 2, KL_SSSSM = 3 };

__host__ __device__ inline int lu_kind_of(int qr_kind)
{
    switch (qr_kind) {
    case K_GEQRT: return KL_GETRF;
    case K_LARFB: return KL_GESSM;
    case K_TSQRT: return KL_TSTRF;
    default: return KL_SSSSM;
    }
}

}  // namespace tqr
