// Device-resident state of one simulator instance and the step kernels.
//
// Layout in HBM (structure of arrays):
//   links   geo[L]   float4 (length, u dt, jam spacing s = dn/kappa, tag band)
//           lst[L]   int4   (queue base slot, queue capacity, q_fx, credit cap)
//           lnode[L] int4   (head node, zone of the head node, choice-set begin/end)
//           tinfo[L] float4 (U = beta/c + w.phi, G = w.psi, head node bits, L/2)
//           lq[L]    int4   (queue head index, queue length, credit, exits) dynamic
//           vac[L]   int    link is vacant for the coming step's node model
//   queues  pos[2][S] float ping-pong positions, svid[S] vehicle of each slot;
//           link j owns slots [qbase_j, qbase_j + qcap_j) used as a ring in
//           FIFO order (leader first): the order of SI-A's argsort, maintained
//           instead of re-sorted because vehicles never overtake.
//   merge   W[2][L] u64 merge words (one buffer per step parity).
//   origins fifo_list[N] vehicles sorted by (origin, departure step, id),
//           fifo_dep[N] their departure steps, fifo_ptr[V] next to release.
#pragma once
#include "ts_device.cuh"

namespace ts {

struct DevSim {
    int V, L, N, Z, F;
    int dn_fx, obs_every;
    float M, eps_arr, dt;
    uint32_t key0, key1;
    // static link data
    const float4 *geo;
    const int4 *lst;
    const int4 *lnode;
    const float4 *tinfo;
    const float *alpha;            // [L + 1]: merge priority; [L] = origin queues
    const int *lo_idx;
    // static node / vehicle data
    const int *no_ptr, *no_idx, *node_zone;
    const int *fifo_end, *fifo_list, *fifo_dep;
    const int *dest_zone;
    const float *dest_feat;
    // dynamic
    int4 *lq;
    int *vac;
    float *pos0, *pos1;
    int *svid;
    unsigned long long *W0, *W1;
    int *cand_vid, *cand_tgt;      // [L]
    int *ncand_vid, *ncand_tgt;    // [V]
    int *fifo_ptr;                 // [V]
    int *entry, *vstate;           // [N]
    float *acc_dx;
    int *acc_n, *tt_sum, *tt_cnt, *C_prev;
    int *out_counts;
    float *out_speed, *out_tt;
    int *step_delta;               // [T][4]: origin releases, arrivals, candidates, entries
    int *err;                      // [4]
    // tape (backward); null when not recording
    int8_t *tag_tape;              // [S] tag of the slot's vehicle in the last step
};

__device__ __forceinline__ void set_error(const DevSim &d, int code, int a, int b) {
    if (atomicCAS(d.err, 0, code) == 0) { d.err[1] = a; d.err[2] = b; }
}

// Observation at time t (SI-D): C_j = exits_j + vehicles past the midpoint;
// closes bin (t-1)/obs_every of counts, speeds and link times.
__device__ __forceinline__ void observe_link(const DevSim &d, int j, int lane, int t, int4 q, int4 st, const float *pc) {
    const float half = d.tinfo[j].w;
    int past = 0;
    for (int k = lane; k < q.y; k += 32) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        past += pc[st.x + idx] >= half;
    }
    past = warp_sum(past);
    if (lane == 0) {
        const int b = (t - 1) / d.obs_every;
        const size_t o = (size_t)b * d.L + j;
        const int C = q.w + past;
        d.out_counts[o] = C - d.C_prev[j];
        d.C_prev[j] = C;
        const int an = d.acc_n[j];
        d.out_speed[o] = an ? d.acc_dx[j] / ((float)an * d.dt) : 0.0f;
        const int tc = d.tt_cnt[j];
        d.out_tt[o] = tc ? (float)d.tt_sum[j] * d.dt / (float)tc : 0.0f;
        d.acc_dx[j] = 0.0f; d.acc_n[j] = 0; d.tt_sum[j] = 0; d.tt_cnt[j] = 0;
    }
}

// Utility + Gumbel key of turning into link m for a vehicle bound for zone z
// (SI-B: V = beta/c + features, argmax of log z + g).
__device__ __forceinline__ float choice_key(const DevSim &d, int m, int z, int vid, int t, int slot) {
    const float4 ti = d.tinfo[m];
    const float df = d.dest_feat[(size_t)z * d.V + __float_as_int(ti.z)];
    const float v = __fadd_rn(ti.x, __fmul_rn(ti.y, df));
    return __fadd_rn(v, gumbel(d.key0, d.key1, vid, t, 0, slot));
}

}  // namespace ts
