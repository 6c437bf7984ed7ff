// release.cuh -- completion of a task in the graph of graph.cuh: the
// successors are signalled cooperatively by all threads of the CTA (the
// mirror of g_ndeps).  Shared by the QR and LU persistent kernels.
#pragma once
#include "graph.cuh"
#include "sched.cuh"

namespace tqr {

// The threads first, first + stride, ... of the CTA take part (default: all).
__device__ static void release_graph(const Queues &Q, const TGraph &G, int kind, int k, int i, int j,
                                     int first = threadIdx.x, int stride = NT)
{
    const int fan = g_fanout(G, kind, k);
    GTask sp[2];
    const int nsp = g_specific(G, kind, k, i, j, sp);
    for (int s = first; s < fan + nsp; s += stride) {
        const GTask t = s < fan ? g_fan_task(kind, k, i, s) : sp[s - fan];
        const int tk = g_kind(G, t.tt, t.k, t.i, t.j);
        q_signal(Q, g_cidx(G, t.tt, t.k, t.i, t.j), g_ndeps(tk, t.k), kind_prio(tk, t.k, t.j),
                 encode_task(t.k, t.i, t.j, t.tt));
    }
}

}  // namespace tqr
