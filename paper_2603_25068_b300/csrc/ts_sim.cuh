// Device-resident state of one simulator instance.
//
// Layout in HBM (structure of arrays):
//   links   geo[L]    float4 (length, u dt, jam spacing s = dn/kappa, tag band)
//           lst[L]    int4   (queue base slot, queue capacity, q_fx, credit cap)
//           lnode[L]  int4   (head node, zone of the head node, choice-set begin/end)
//           tinfo[L]  float4 (U = beta/c + w.phi, G = w.psi, head node bits, L/2)
//   blocks  blk_links[] links [blk_links[b], blk_links[b+1]) form link block b of
//           k_step_a (queue capacities packed up to the shared-memory stage)
//           lq[L]     int4   (queue head index, queue length, credit, exits) dynamic
//           crec[L]   int4   (candidate vehicle, target, entry step << 8 | next-step
//                            vacancy/arrival bits, leader's new position)
//           vac[L]    int    link is vacant for the coming step's node model
//   choice  loinfo[E] float4 (U, G, head bits, link bits) of every choice-set entry;
//           noinfo[E'] the same for the out-links of every node (origin queues)
//   queues  pos[2][S] float ping-pong positions; saux[S] int2 (vehicle, destination
//           zone); sentry[S] entry step.  Link j owns slots [qbase_j, qbase_j +
//           qcap_j), used as a ring in FIFO order (leader first): the order of
//           SI-A's argsort, maintained instead of re-sorted because vehicles never
//           overtake.
//   merge   W[2][L] u64 merge words (one buffer per step parity).
//   origins fifo_list[N] vehicles sorted by (origin, departure step, id),
//           fifo_dep[N] their departure steps, fifo_ptr[V] next to release,
//           nrec[V] int2 (candidate vehicle, target).
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
    const int *ebits;              // [L] next-step vacancy/arrival bits of an empty link (from geo)
    const int4 *lst;
    const int4 *lnode;
    const float4 *tinfo;
    const float *alpha;            // [L + 1]: merge priority; [L] = origin queues
    const float4 *loinfo;
    const int *blk_links;          // [nblk + 1] first link of each block of k_step_a
    int nblk;                      // blocks of k_step_a
    int npb;                       // origin queues per block of k_step_a
    // static node / vehicle data
    const int *no_ptr, *node_zone;
    const float4 *noinfo;
    const int *fifo_end, *fifo_dep;
    const int2 *fifo_list;         // [N] (vehicle, destination zone) in queue order
    const int *dest_zone;
    const float *dest_feat;
    // dynamic
    int4 *lq;
    int4 *crec;
    int *vac;
    float *pos0, *pos1;
    int2 *saux;                    // [S] (vehicle, destination zone)
    int *sentry;                   // [S] entry step of the slot's vehicle
    unsigned long long *W0, *W1;
    int2 *nrec;                    // [V] origin-queue candidate (vehicle, target)
    int *fifo_ptr;                 // [V]
    int *vstate;                   // [N] link, or waiting / arrived
    int4 *lstat;                   // [L] (vehicle-steps, link-time sum, leavers, C_prev) of the open bin
    longlong2 *lpos;               // [L] (position sum at bin start, leavers' positions), 2^-16 m
    int *out_counts;
    float *out_speed, *out_tt;
    int *step_delta;               // [T][4]: origin releases, arrivals, candidates, entries
    int *err;                      // [4]
    // tape (backward); null when not recording
    int8_t *tag_tape;              // [S] car-following tag of each slot's vehicle this step
    float *tape_pos;               // [S] positions at the start of this step (occupied slots;
                                   // recorded at bin ends only)
    int *tape_vid;                 // [S] vehicle of each occupied slot at the start of the
                                   // segment (written at its first step only; null after)
    int *tape_ent;                 // [L tape_K] entrant log of the segment: entrant m of link j
                                   // (counted from the segment start) at j tape_K + m
    const int4 *tape_lq0;          // [L] queue states at the start of the segment
    int tape_K;                    // steps of a segment
    int4 *tape_lq;                 // [L] queue state at the start of this step
    int4 *tape_crec;               // [L] link records of this step
    int2 *tape_nrec;               // [V] origin-queue records of this step
    unsigned long long *tape_W;    // [L] merge words of this step
    float *tape_mkey;              // [L + V] merge key alpha + g' of each candidate with a
                                   // target this step (links, then origin queues)
    int2 *route_log;               // [N * route_cap] (step, link) of every entry; null = off
    int *route_len;                // [N] entries so far
    int route_cap;
};

__device__ __forceinline__ void set_error(const DevSim &d, int code, int a, int b) {
    if (atomicCAS(d.err, 0, code) == 0) { d.err[1] = a; d.err[2] = b; }
}

}  // namespace ts
