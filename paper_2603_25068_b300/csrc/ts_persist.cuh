// Persistent forward executor (sm_103a): a run of steps in ONE cooperative
// launch, one CTA of kPT threads per SM, each CTA owning a fixed group of
// consecutive links and a fixed range of origin queues for the whole launch.
//
// The queues of a CTA's links stay in its shared memory for the whole launch
// (FIFO rings, leader first, one float position per slot: the order of SI-A's
// argsort, maintained instead of re-sorted because vehicles never overtake), so
// that the car-following update reads and writes no global memory.  The
// (vehicle, zone, entry step) of the first two queue positions of every link
// and of every origin queue are cached in shared memory too, so that finding
// the candidates of a step loads nothing.  Across CTAs, the node model of SI-B
// couples links only through
//   * the merge words W[target] (64-bit atomicMax of alpha + g' over the
//     candidates, low half ~(vehicle << 8 | zone) when the sizes allow, so that
//     the target learns the entrant's zone with the word), three buffers
//     indexed by step mod 3; the owner of a link that is not vacant at the
//     step stores kWBlocked in its word, which no candidate's word exceeds,
//     so that the word carries the link's vacancy too.
// A candidate is valid when its chosen link is vacant (SI-B: a link accepts
// an entrant only if its rearmost vehicle has left the jam spacing), and every
// candidate of one target shares that target's vacancy.  So the validity test
// is taken where the merge is resolved, one step later: every candidate
// takes part in the atomicMax of its chosen link; in the transfers of step t
// the owner of a link admits the word's winner only if the link was vacant at
// t, and the owner of a candidate pops it only if it won and its target was
// vacant (both read from the target's word, in one load).  Merges, winners
// and transfers are exactly those of the per-step definition, while the choice
// phase loads nothing but the destination features.  One grid-wide barrier per
// step therefore suffices.  Epoch t of a CTA:
//   T   transfers of step t-1 for its links and origin queues (one round of
//       merge-word loads), its links' vacancy at t stored into their words of
//       step t, the car-following of each link's first two vehicles and its
//       entrant, then credit and candidates of step t and the warp ballots of
//       the step counters;
//   S   one block scan: the compact list of (candidate, choice slot) pairs and
//       each link's first vehicle in the CTA's order of the vehicles that the
//       car-following runs take;
//   C   every warp evaluates pairs (utility + Gumbel key of each slot, the
//       merge key); the last warp adds up the step counters;
//   P   argmax, merge atomicMax and records (link and origin-queue threads),
//       beside them the next-step bits and the runs' first links (warps that
//       hold neither); then the last warp's arrival at the grid barrier;
//   W   while that warp polls, threads 0 .. kPCF - 1 run the car-following of
//       step t + 1 for queue positions >= 2 (their vehicle ahead stays
//       whatever the transfers do).
//
// Every floating-point operation is the one of the two-kernel path (same device
// functions, same order), so both executors give bit-identical results.
// Every wait is bounded: a barrier that does not complete within ~2 s records
// SIM_ETIMEOUT and every CTA returns.
#pragma once
#include "ts_step.cuh"

namespace ts {

constexpr int kPT = 1024;                    // threads per CTA
constexpr int kPLinks = 288;                 // links per CTA at most
constexpr int kPNodes = 128;                 // origin queues per CTA at most
constexpr int kPNodeTid = 512;               // thread of origin queue 0 in the per-entity phases
constexpr int kPSlot = 8;                    // choice slots per candidate evaluated in parallel
// The last warp takes no part in the car-following: its first thread makes the
// CTA's arrival at the grid barrier (whose release ordering waits until the
// CTA's writes are performed) and then polls, while threads 0 .. kPCF - 1 run
// the car-following of the barrier wait without waiting for that ordering.
constexpr int kPCF = kPT - 32;               // car-following threads
constexpr int kPBarTid = kPCF;               // thread of the grid barrier's arrival and wait
constexpr int kPBitsTid = 640;               // thread of link 0 in p_bits (warps with no link or origin queue)
constexpr int kPEnt = kPLinks + kPNodes;     // entities: links, then origin queues (index kPLinks + node)
constexpr int kPPairs = kPEnt * (kPSlot + 1);
static_assert(kPSlot + 1 <= 16, "a pair list entry holds the slot in 4 bits");
static_assert(kPNodeTid >= kPLinks && kPBitsTid >= kPNodeTid + kPNodes && kPBitsTid + kPLinks <= kPCF &&
              kPBitsTid % 32 == 0, "link, origin-queue, next-step-bit and barrier threads are disjoint warps");

struct PArgs {
    const int *grp_links;          // [G + 1] first link of each CTA's group
    int npg;                       // origin queues per CTA
    int packz;                     // merge words carry the entrant's zone
    unsigned long long *W3;        // [3 L] merge words by step mod 3 (kWBlocked: the link is not vacant)
    unsigned *bar;                 // grid barrier counter (zero at launch)
    int t0, t1;                    // steps [t0, t1)
    int final_obs;                 // close the last bin at t1 (observation-only pass)
    int S;                         // tape stride of the slot records (recording launches)
    int bar_extra;                 // arrivals the first barrier waits for beyond the grid (0; > 0 in
                                   // tests of the bounded wait: they never come)
    uint32_t rk[2][10];            // Philox round keys: key0 + r 0x9E3779B9, key1 + r 0xBB67AE85 (mod 2^32)
    int skip2;                     // barrier-wait runs over queue positions >= 2 only (long queues)
};

// Merge word of a link that is not vacant at the step: stored by the link's
// owner in the transfers that settle the vacancy, before or after the
// candidates' max reductions of the step (the maximum is the same either way:
// a real word has a float key in its high half, never all ones).
constexpr unsigned long long kWBlocked = ~0ull;

struct PSmem {
    int4 q[kPLinks];               // queue head, length, credit, exits
    int4 st[kPLinks];              // global slot base, capacity, q_fx, credit cap
    float4 g[kPLinks];             // length, u dt, s, tag band
    int4 nd[kPLinks];              // head node, head zone, first staged choice entry, choice count
    int4 stat[kPLinks];            // open-bin statistics
    int4 cr[kPLinks];              // record of the step (candidate, target, entry << 8 | bits, x0)
    int4 ld[kPLinks];              // (vehicle, zone) at queue positions 0 and 1
    int2 le[kPLinks];              // entry steps at queue positions 0 and 1
    int flags[kPLinks];            // vacancy / arrival for the coming step
    int e0[kPLinks];               // recording: entries (exits + queued) at the segment start
    int lbase[kPLinks + 1];        // first ring slot of each link in shared memory (static)
    int voff[kPLinks + 1];         // first vehicle of each link in the CTA's queue order (step t)
    int past[kPLinks];             // bin end: vehicles past the midpoint (time t), summed over the step
    float xt[kPLinks];             // position of the rearmost vehicle after the step's car-following
    int nbits[kPLinks];            // next-step vacancy / arrival bits of the link record (p_bits)
    int cfli[kPCF];                // link of the first vehicle of each car-following run (p_run_links)
    float mkey[kPEnt];              // merge key alpha + g' of each entity's candidate
    float alpha[kPLinks];
    unsigned long long psum[kPLinks];
    float key[kPSlot][kPEnt];      // key of choice slot k of each entity's candidate (slot-major: no bank conflicts)
    int tv[kPSlot][kPEnt];         // link of choice slot k
    longlong2 lpos[kPLinks];       // position sums of the open bin: at its start, of its leavers (2^-16 m)
    int4 nq[kPNodes];              // next vehicle, end of queue, first staged out-link entry, out-degree
    int4 nh[kPNodes];              // (vehicle, zone) at queue positions 0 and 1
    int2 ndep[kPNodes];            // departure steps at queue positions 0 and 1
    int2 nrec[kPNodes];            // (candidate, target) of the step
    int nzone[kPNodes];
    int plist[kPPairs];            // entity << 4 | (0 merge key, 1 + k choice slot k)
    int wsum[32];
    int cnt[4];                    // step counters: releases, arrivals, candidates, entries
    unsigned cbal[4][kPT / 32];    // the same counters of the step as one ballot per warp
    int npairs, ctot, stop;
};

// Shared-memory bytes of a CTA beyond PSmem: ring slots, staged choice records
// of its links and of its origin nodes' out-links (16-byte aligned sections).
__host__ __device__ inline size_t p_dyn_bytes(long long slots, long long n_lo, long long n_no) {
    return (((size_t)slots * 4 + 15) & ~(size_t)15) + (size_t)(n_lo + n_no) * 16;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// merge reduction with no value returned: the thread does not wait for it
__device__ __forceinline__ void red_max_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number `target / gridDim.x` (counter never reset inside a
// launch), in two halves so that a CTA can work between its arrival and the
// wait: grid_arrive (block barrier, then one release arrival by thread
// kPBarTid) and grid_wait (polled by the same thread).
// Bounded: gives up after ~2 s or 2^22 polls, or as soon as another CTA has
// recorded a timeout; returns false then (every thread of the CTA).
__device__ __forceinline__ void grid_arrive(unsigned *bar) {
    __syncthreads();
    // release arrival: covers this CTA's writes ordered before it by the block
    // barrier; the acquire load that sees the target covers the rest
    if (threadIdx.x == kPBarTid) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(bar) : "memory");
}
__device__ __forceinline__ bool grid_wait(const DevSim &d, unsigned *bar, unsigned target, int t, int *stop) {
    // thread kPBarTid waits as soon as it has arrived; the block barrier after
    // the wait holds every thread until both its own work and the grid's are
    if (threadIdx.x == kPBarTid) {
        const unsigned long long t_start = global_ns();
        int ok = 1;
        for (unsigned it = 0;; ++it) {
            if (ld_acquire_gpu(bar) >= target) break;
            if ((it & 255u) == 255u) {
                if (it >= (1u << 22) || global_ns() - t_start > 2000000000ull ||
                    __ldcg(d.err) == SIM_ETIMEOUT) {
                    set_error(d, SIM_ETIMEOUT, (int)blockIdx.x, t);
                    ok = 0;
                    break;
                }
            }
        }
        *stop = !ok;
    }
    __syncthreads();
    return *stop == 0;
}
__device__ __forceinline__ bool grid_sync(const DevSim &d, unsigned *bar, unsigned target, int t, int *stop) {
    grid_arrive(bar);
    return grid_wait(d, bar, target, t, stop);
}

// merge words: the key in the high half; ~(vehicle << 8 | zone) or ~vehicle in
// the low half (the largest key wins, equal keys go to the lowest vehicle)
__device__ __forceinline__ unsigned long long p_word(float key, int vid, int zone, int packz) {
    if (!packz) return merge_word(key, vid);
    const unsigned long long w = merge_word(key, 0);
    return (w & 0xffffffff00000000ull) | (unsigned long long)(~(((uint32_t)vid << 8) | (uint32_t)zone));
}
__device__ __forceinline__ int p_vid(unsigned long long w, int packz) {
    return packz ? (int)((~(uint32_t)(w & 0xffffffffull)) >> 8) : merge_vid(w);
}

// Philox4x32-10 with the key schedule read from the launch's parameters
// (a.rk): the same function as philox4x32_10(c, key0, key1), without the two
// key additions of each round.  The Gumbel draw of (vehicle, step, stream,
// slot) as gumbel() gives it.
__device__ __forceinline__ uint4 p_philox(const PArgs &a, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;   // one wide multiply each
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ a.rk[0][r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ a.rk[1][r],
                       (uint32_t)p0);
    }
    return c;
}
__device__ __forceinline__ float p_gumbel(const PArgs &a, int vid, int t, int stream, int slot) {
    const uint4 o = p_philox(a, make_uint4((uint32_t)vid, (uint32_t)t, (uint32_t)stream, (uint32_t)(slot >> 2)));
    const int s = slot & 3;
    return gumbel_of_word(s == 0 ? o.x : s == 1 ? o.y : s == 2 ? o.z : o.w);
}

// argmax of the staged keys (ties to the lowest slot); slots past the stage
// are evaluated inline.  Returns the chosen link (its vacancy is taken at the
// transfers).
__device__ __forceinline__ int p_choose(const DevSim &d, const PSmem &S, int ei, const float4 *info, int deg,
                                        int zone, int vid, int t) {
    float bk = -INFINITY;
    int bm = -1;
#pragma unroll
    for (int k = 0; k < kPSlot; ++k) {
        if (k < deg) {
            const float kk = S.key[k][ei];
            const int m = S.tv[k][ei];
            if (bm < 0 || kk > bk) { bk = kk; bm = m; }
        }
    }
    for (int k = kPSlot; k < deg; ++k) {
        const float4 e = info[k];
        const float kk = choice_key(d, e, zone, vid, t, k);
        if (kk > bk) { bk = kk; bm = __float_as_int(e.w); }
    }
    return bm;
}

// A refill of the second cached queue position, loaded in phase T and stored
// after the other phases (its value is needed only at the next pop).
struct PPend {
    int2 aux;
    int ent;
    int on;
};

__device__ __forceinline__ int2 ld_int2(const int2 *p) {
    int2 v;
    asm volatile("ld.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_int(const int *p) {
    int v;
    asm volatile("ld.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

struct PCtx {
    int j0, nl, n0, nn, base0, nslots;
    float *P;                      // ring slots
    const float4 *LO;              // staged choice records of the links
    const float4 *NO;              // staged out-link records of the origin nodes
    int lo0, no0;                  // first staged entry (global index)
};

// Car-following of step t (SI-A) for the vehicles of link li whose update the
// transfers of step t - 1 decide: the old leader if it stays (headway M), the
// second vehicle (the leader if the first one leaves) and the entrant at x = 0
// (behind the old rearmost vehicle, whose time-t position p_decide kept in
// S.xt).  q0 is the queue before the transfers; the other vehicles were
// updated during the grid barrier before (p_carfollow with kMin = 2).  The
// updates of both outcomes are computed first (p_ends_pre, while the loads of
// the merge words are in flight), then the outcome picks (p_ends_post).  At
// bin ends the time-t positions join the link's sums.
struct PEnds {
    float x0, x1, y0, y1m, y1f, yem, yet;
    int tags;                      // 2 bits each: y0, y1m, y1f, yem, yet
};

__device__ __forceinline__ PEnds p_ends_pre(const DevSim &d, const PSmem &S, const PCtx &c, int li, int4 q0) {
    const float M = d.M;
    const float4 g = S.g[li];
    const int4 st = S.st[li];
    const int lb = st.x - c.base0, cap = st.y, n = q0.y;
    const int i1 = q0.x + 1 >= cap ? q0.x + 1 - cap : q0.x + 1;
    PEnds e;
    e.x0 = n >= 1 ? c.P[lb + q0.x] : 0.0f;
    e.x1 = n >= 2 ? c.P[lb + i1] : 0.0f;
    int t0, t1, t2, t3, t4;
    e.y0 = newell(e.x0, M, g.x, g.y, g.z, g.w, t0);
    e.y1m = newell(e.x1, M, g.x, g.y, g.z, g.w, t1);
    e.y1f = newell(e.x1, __fsub_rn(e.x0, e.x1), g.x, g.y, g.z, g.w, t2);
    e.yem = newell(0.0f, M, g.x, g.y, g.z, g.w, t3);
    e.yet = newell(0.0f, __fsub_rn(S.xt[li], 0.0f), g.x, g.y, g.z, g.w, t4);
    e.tags = t0 | (t1 << 2) | (t2 << 4) | (t3 << 6) | (t4 << 8);
    return e;
}

template <bool kTape>
__device__ __forceinline__ void p_ends_post(const DevSim &d, const PArgs &a, PSmem &S, const PCtx &c, int li,
                                            int4 q0, const PEnds &e, bool pop, bool push, int t, bool obs) {
    const int4 st = S.st[li];
    const int lb = st.x - c.base0, cap = st.y, n = q0.y;
    const int i0 = q0.x, i1 = q0.x + 1 >= cap ? q0.x + 1 - cap : q0.x + 1;
    int ie = q0.x + n;
    if (ie >= cap) ie -= cap;
    const bool up0 = n >= 1 && !pop, up1 = n >= 2;
    const bool lead_e = n == 0 || (pop && n == 1);          // the entrant is alone on the link
    if (obs) {
        const float half = __fmul_rn(S.g[li].x, 0.5f);
        int past = 0;
        long long ps = 0;
        if (up0) { past += e.x0 >= half ? 1 : 0; ps += pos_fx(e.x0); }
        if (up1) { past += e.x1 >= half ? 1 : 0; ps += pos_fx(e.x1); }
        S.past[li] += past;                                   // the entrant at 0 adds nothing
        S.psum[li] += (unsigned long long)ps;
    }
    if (up0) c.P[lb + i0] = e.y0;
    if (up1) c.P[lb + i1] = pop ? e.y1m : e.y1f;
    if (push) c.P[lb + ie] = lead_e ? e.yem : e.yet;
    if (kTape) {                    // tape: branch tag of the slot, time-t position at bin ends
        const size_t o = (size_t)(t - a.t0) * a.S + c.base0 + lb;
        if (up0) d.tag_tape[o + i0] = (int8_t)(e.tags & 3);
        if (up1) d.tag_tape[o + i1] = (int8_t)((e.tags >> (pop ? 2 : 4)) & 3);
        if (push) d.tag_tape[o + ie] = (int8_t)((e.tags >> (lead_e ? 6 : 8)) & 3);
        if (obs) {
            if (up0) d.tape_pos[o + i0] = e.x0;
            if (up1) d.tape_pos[o + i1] = e.x1;
            if (push) d.tape_pos[o + ie] = 0.0f;
        }
    }
}

// Transfers of step tb for this thread's link or origin queue (SI-B Eq.
// transfer): pop the leader that won its merge into a vacant link or left to its
// destination, push the merge winner at x = 0 if the link was vacant at tb,
// flags of step tb + 1 and their publication.  The record of step tb gets its
// final target (kTgtBlocked when the chosen link was not vacant).  Counters
// accumulate.
template <bool kTape>
__device__ __forceinline__ void p_apply(const DevSim &d, const PArgs &a, PSmem &S, const PCtx &c, int tb, PPend &pd,
                                        int *cnt, bool cf, bool obs) {
    const int tid = threadIdx.x;
    const unsigned long long *Wb = a.W3 + (size_t)(tb % 3) * d.L;
    unsigned long long *Wn = a.W3 + (size_t)((tb + 1) % 3) * d.L;   // words of step tb + 1 (vacancy)
    if (tid < c.nl) {
        const int li = tid, j = c.j0 + li;
        int4 q = S.q[li];
        const int4 st = S.st[li];
        int4 cr = S.cr[li];
        const unsigned long long w0 = __ldcg(Wb + j);
        cr.z |= S.nbits[li];                                 // the record's next-step bits
        unsigned long long wt = 0ull;
        if (cr.y >= 0) wt = __ldcg(Wb + cr.y);             // the target's word and its vacancy
        PEnds ends;
        if (cf) ends = p_ends_pre(d, S, c, li, q);            // while the loads are in flight
        // the candidates of a link that was not vacant at tb could not enter it:
        // its word names no entrant
        const unsigned long long win = (S.flags[li] & kFlagVacant) ? w0 : 0ull;
        if (kTape)                  // the tape keeps merge words in the standard format (~vehicle low half)
            d.tape_W[(size_t)(tb - a.t0) * d.L + j] =
                win ? ((win & 0xffffffff00000000ull) | (unsigned long long)(~(uint32_t)p_vid(win, a.packz))) : 0ull;
        bool pop = false;
        cnt[2] += cr.x >= 0;
        if (cr.y == kTgtSink) {
            pop = true;
            d.vstate[cr.x] = kVehArrived;
            cnt[1] += 1;
        } else if (cr.y >= 0) {
            if (wt != kWBlocked) pop = wt != 0ull && p_vid(wt, a.packz) == cr.x;
            else cr.y = kTgtBlocked;
        }
        if (kTape) d.tape_crec[(size_t)(tb - a.t0) * d.L + j] = cr;
        S.cr[li] = cr;
        const int4 q0 = q;                                   // the queue before the transfers
        int4 ld = S.ld[li];
        int2 le = S.le[li];
        if (pop) {
            int4 stat = S.stat[li];
            stat.y += tb + 1 - (cr.z >> 8);
            stat.z += 1;
            S.stat[li] = stat;
            S.lpos[li].y += pos_fx(__int_as_float(cr.w));
            q.x = (q.x + 1 == st.y) ? 0 : q.x + 1;
            q.y -= 1;
            q.z -= d.dn_fx;
            q.w += 1;
            ld.x = ld.z;
            ld.y = ld.w;
            le.x = le.y;
            if (q.y >= 2) {
                int idx = q.x + 1;
                if (idx >= st.y) idx -= st.y;
                pd.aux = ld_int2(d.saux + st.x + idx);
                pd.ent = ld_int(d.sentry + st.x + idx);
                pd.on = 1;
            }
        }
        bool push = win != 0ull;
        if (push) {
            const int v = p_vid(win, a.packz);
            if (q.y >= st.y) {
                set_error(d, SIM_EOVERFLOW, j, tb);
                push = false;
            } else {
                const int z = a.packz ? (int)((~(uint32_t)(win & 0xffffffffull)) & 0xffu) : d.dest_zone[v];
                int idx = q.x + q.y;
                if (idx >= st.y) idx -= st.y;
                c.P[st.x - c.base0 + idx] = 0.0f;
                d.saux[st.x + idx] = make_int2(v, z);
                d.sentry[st.x + idx] = tb + 1;
                if (kTape) {                // entrant log of the segment (reverse pass)
                    const int m = q.w + q.y - S.e0[li];
                    if (m >= 0 && m < d.tape_K) d.tape_ent[(size_t)j * d.tape_K + m] = v;
                    else set_error(d, SIM_EOVERFLOW, j, tb);
                }
                if (q.y == 0) { ld.x = v; ld.y = z; le.x = tb + 1; }
                if (q.y == 1) { ld.z = v; ld.w = z; le.y = tb + 1; }
                q.y += 1;
                d.vstate[v] = j;
                cnt[3] += 1;
                if (d.route_log) {
                    const int r = d.route_len[v];
                    if (r < d.route_cap) {
                        d.route_log[(size_t)v * d.route_cap + r] = make_int2(tb, j);
                        d.route_len[v] = r + 1;
                    } else {
                        set_error(d, SIM_EOVERFLOW, -1 - v, tb);
                    }
                }
            }
        }
        if (cf) p_ends_post<kTape>(d, a, S, c, li, q0, ends, pop, push, tb + 1, obs);
        S.q[li] = q;
        S.ld[li] = ld;
        S.le[li] = le;
        const int o = (pop ? 1 : 0) | (push ? 2 : 0);
        const int fl = ((cr.z >> o) & 1) | (((cr.z >> (4 + o)) & 1) << 1);
        S.flags[li] = fl;
        if (!(fl & kFlagVacant)) Wn[j] = kWBlocked;         // read by the transfers of step tb + 1
        a.W3[(size_t)((tb + 2) % 3) * d.L + j] = 0ull;      // words of step tb + 2 start from zero
    } else if (tid >= kPNodeTid && tid < kPNodeTid + c.nn) {
        const int ni = tid - kPNodeTid;
        int2 cr = S.nrec[ni];
        cnt[2] += cr.x >= 0;
        bool rel = false;
        if (cr.y == kTgtSink) {
            rel = true;
            d.vstate[cr.x] = kVehArrived;
            cnt[1] += 1;
        } else if (cr.y >= 0) {
            const unsigned long long w = __ldcg(Wb + cr.y);
            if (w != kWBlocked) rel = w != 0ull && p_vid(w, a.packz) == cr.x;
            else cr.y = kTgtBlocked;
        }
        if (kTape) d.tape_nrec[(size_t)(tb - a.t0) * d.V + c.n0 + ni] = cr;
        S.nrec[ni] = cr;
        if (rel) {
            cnt[0] += 1;
            int4 nq = S.nq[ni];
            int4 nh = S.nh[ni];
            int2 dp = S.ndep[ni];
            nq.x += 1;
            nh.x = nh.z;
            nh.y = nh.w;
            dp.x = dp.y;
            if (nq.x + 1 < nq.y) {
                pd.aux = ld_int2(d.fifo_list + nq.x + 1);
                pd.ent = ld_int(d.fifo_dep + nq.x + 1);
                pd.on = 1;
            }
            S.nq[ni] = nq;
            S.nh[ni] = nh;
            S.ndep[ni] = dp;
        }
    }
}

// the refill loaded by p_apply (second queue position)
__device__ __forceinline__ void p_refill(PSmem &S, const PCtx &c, const PPend &pd) {
    if (!pd.on) return;
    const int tid = threadIdx.x;
    if (tid < c.nl) {
        S.ld[tid].z = pd.aux.x;
        S.ld[tid].w = pd.aux.y;
        S.le[tid].y = pd.ent;
    } else {
        const int ni = tid - kPNodeTid;
        S.nh[ni].z = pd.aux.x;
        S.nh[ni].w = pd.aux.y;
        S.ndep[ni].y = pd.ent;
    }
}

// add this thread's step counters to the CTA's (every thread calls)
__device__ __forceinline__ void p_count(PSmem &S, const int *cnt) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int v = (int)__reduce_add_sync(kFull, (unsigned)cnt[k]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&S.cnt[k], v);
    }
}

// The same counters as ballots, one word per warp and counter (a thread's
// transfers add at most one to each: one link or origin queue per thread).
// Every thread calls; p_count_sum adds them up later, off the phases' path.
__device__ __forceinline__ void p_count_bal(PSmem &S, const int *cnt) {
    const int w = threadIdx.x >> 5;
    const unsigned b0 = __ballot_sync(kFull, cnt[0] != 0), b1 = __ballot_sync(kFull, cnt[1] != 0);
    const unsigned b2 = __ballot_sync(kFull, cnt[2] != 0), b3 = __ballot_sync(kFull, cnt[3] != 0);
    if ((threadIdx.x & 31) == 0) {
        S.cbal[0][w] = b0;
        S.cbal[1][w] = b1;
        S.cbal[2][w] = b2;
        S.cbal[3][w] = b3;
    }
}
// the CTA's counters of step tb from the ballots, added to the step's deltas
// (one whole warp calls)
__device__ __forceinline__ void p_count_sum(const DevSim &d, const PSmem &S, int tb) {
    const int lane = threadIdx.x & 31;
    int x = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int v = (int)__reduce_add_sync(kFull, (unsigned)__popc(S.cbal[k][lane]));
        if (lane == k) x = v;
    }
    if (lane < 4 && x) atomicAdd(&d.step_delta[4 * tb + lane], x);
}

// Step t of this thread's link or origin queue up to the choice: credit,
// candidate.  Returns (choice pairs (merge key + choice slots) << 16) | the
// link's number of queued vehicles.
template <bool kTape>
__device__ __forceinline__ int p_candidate(const DevSim &d, PSmem &S, const PCtx &c, int t, int r, bool obs_only,
                                           bool all = true) {
    const int tid = threadIdx.x;
    if (tid < c.nl) {
        const int li = tid;
        const int4 q = S.q[li];
        // vehicles the car-following runs of the step take: every one (all),
        // else those at queue positions >= 2 (the barrier-wait runs)
        const int cost = all ? q.y : max(q.y - 2, 0);
        if (obs_only) return cost;
        if (kTape) {
            d.tape_lq[(size_t)r * d.L + c.j0 + li] = q;
            if (r == 0) S.e0[li] = q.w + q.y;
        }
        const int4 st = S.st[li];
        const int credit = min(q.z + st.z, st.w);
        S.q[li].z = credit;
        const bool cand = q.y > 0 && (S.flags[li] & kFlagArrive) && credit >= d.dn_fx;
        const int4 nd = S.nd[li];
        const int4 ld = S.ld[li];
        S.cr[li] = make_int4(cand ? ld.x : -1, kTgtNone, cand ? S.le[li].x : 0, 0);
        return (((cand && nd.y != ld.y) ? 1 + min(nd.w, kPSlot) : 0) << 16) | cost;
    }
    if (!obs_only && tid >= kPNodeTid && tid < kPNodeTid + c.nn) {
        const int ni = tid - kPNodeTid;
        const int4 nq = S.nq[ni];
        const int4 nh = S.nh[ni];
        const bool cand = nq.x < nq.y && S.ndep[ni].x <= t;
        S.nrec[ni] = make_int2(cand ? nh.x : -1, kTgtNone);
        return ((cand && S.nzone[ni] != nh.y) ? 1 + min(nq.w, kPSlot) : 0) << 16;
    }
    return 0;
}

// Block scan of every thread's (choice pairs << 16 | queued vehicles): the
// compact pair list and the first vehicle of each link in the CTA's queue
// order (the queues of its links one after another, leader first), from which
// the car-following threads take equal runs of vehicles.
__device__ __forceinline__ void p_scan(PSmem &S, const PCtx &c, int v) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, s, o);
        if (lane >= o) s += y;
    }
    if (lane == 31) S.wsum[w] = s;
    __syncthreads();
    if (w == 0) {
        const int x = lane < kPT / 32 ? S.wsum[lane] : 0;  // only the block's warps wrote a total
        int r = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, r, o);
            if (lane >= o) r += y;
        }
        S.wsum[lane] = r - x;
        if (lane == 31) {
            S.npairs = r >> 16;
            S.voff[c.nl] = r & 0xffff;
        }
    }
    __syncthreads();
    const int ex = s - v + S.wsum[w];
    if (tid < c.nl) S.voff[tid] = ex & 0xffff;
    const int np = v >> 16;
    for (int k = 0; k < np; ++k) S.plist[(ex >> 16) + k] = (tid << 4) | k;
    __syncthreads();
}

// The (candidate, slot) pairs, one per thread at a time: slot 0 is the
// candidate's merge key alpha + g' (Gumbel word of stream 1, block 0), slot
// 1 + k the utility + Gumbel key of choice slot k (stream 0, word k of the
// candidate's blocks).  Both kinds run one code path (one Philox block, one
// Gumbel transform), so a warp holding both does not serialise them; the only
// global load is the destination feature of a slot's link, issued before the
// Gumbel draw is computed.
__device__ __forceinline__ void p_pairs(const DevSim &d, const PArgs &a, PSmem &S, const PCtx &c, int t) {
    const int np = S.npairs;
    for (int p = threadIdx.x; p < np; p += kPT) {
        const int e = S.plist[p];
        const int en = e >> 4, sl = e & 15;
        const bool isl = en < kPNodeTid;
        const int ni = en - kPNodeTid;
        const int ei = isl ? en : kPLinks + ni;
        const int4 who = isl ? S.ld[en] : S.nh[ni];
        const int k = sl - 1;
        float4 info = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float df = 0.0f;
        if (sl > 0) {
            info = isl ? c.LO[S.nd[en].z + k] : c.NO[S.nq[ni].z + k];
            df = d.dest_feat[(size_t)who.y * d.V + __float_as_int(info.z)];
        }
        const float g = p_gumbel(a, who.x, t, sl == 0 ? 1 : 0, sl == 0 ? 0 : k);
        if (sl == 0) {
            S.mkey[ei] = __fadd_rn(isl ? S.alpha[en] : d.alpha[d.L], g);
        } else {
            S.key[k][ei] = __fadd_rn(__fadd_rn(info.x, __fmul_rn(info.y, df)), g);
            S.tv[k][ei] = __float_as_int(info.w);
        }
    }
}

// Newell car-following of the queued vehicles of the CTA, in shared memory, by
// threads 0 .. NT - 1 (NT = kPCF; the other threads return at once).  The CTA's vehicles, taken in queue order link after
// link (leader first), are cut into NT equal runs; thread c updates run c one
// vehicle after another, walking from link to link.  The headway of a vehicle
// uses the time-t position of the one ahead: within a run the thread keeps it
// from the previous iteration; for the first vehicle of a run that is not a
// leader it is read before a barrier of the NT threads, after which they
// write.  A slot is written by one thread only.  Queue positions below kMin
// are read but not updated (kMin = 2: the vehicles whose update the coming
// transfers decide, see p_ends_pre).  At bin ends the threads also sum each
// link's vehicles past the midpoint and their positions over the updated
// vehicles (shared-memory atomics: a link may span several runs).
template <bool kTape, bool kObsOnly, int kMin, bool kSkip = false>
__device__ __forceinline__ void p_carfollow(const DevSim &d, const PArgs &a, PSmem &S, const PCtx &c, int r, bool obs) {
    constexpr int NT = kPCF;
    const int ct = threadIdx.x;
    if (ct >= NT) return;
    const float M = d.M;
    const int nv = S.voff[c.nl];                             // < 2^16: ct nv fits in 32 bits
    const int v0 = (ct * nv) / NT, v1 = ((ct + 1) * nv) / NT;
    int li = 0, k = 0, idx = 0, n = 0, lb = 0, cap = 0;
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float ahead = M;
    if (v0 < v1) {
        // the link holding vehicle v0: the last li with voff[li] <= v0 (empty
        // links before it share its offset; those after it start beyond v0),
        // listed by p_run_links for the barrier-wait runs
        if (kMin == 2) {
            li = S.cfli[ct];
        } else {
            int lo = 0, hi = c.nl - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.voff[mid] <= v0) lo = mid; else hi = mid - 1;
            }
            li = lo;
        }
        // kSkip: the offsets count the vehicles at queue positions >= 2 only
        k = v0 - S.voff[li] + (kSkip ? 2 : 0);
        const int2 qv = *reinterpret_cast<const int2 *>(&S.q[li]);
        n = qv.y;
        lb = S.lbase[li];
        cap = S.lbase[li + 1] - lb;
        g = S.g[li];
        idx = qv.x + k;
        if (idx >= cap) idx -= cap;
        if (k > 0) ahead = c.P[lb + (idx == 0 ? cap - 1 : idx - 1)];
    }
    asm volatile("bar.sync 1, %0;" :: "n"(NT) : "memory");         // every run has read its vehicle ahead
    int past = 0;
    long long psum = 0;
    for (int v = v0; v < v1; ++v) {
        if (k == n) {                       // the run continues with the leader of the next occupied link
            if (obs) {
                atomicAdd(&S.past[li], past);
                atomicAdd(&S.psum[li], (unsigned long long)psum);
                past = 0;
                psum = 0;
            }
            do { ++li; } while (S.voff[li + 1] == S.voff[li]);
            const int2 qv = *reinterpret_cast<const int2 *>(&S.q[li]);
            n = qv.y;
            lb = S.lbase[li];
            cap = S.lbase[li + 1] - lb;
            g = S.g[li];
            idx = qv.x;
            k = 0;
            if (kSkip) {                    // from queue position 2, behind position 1
                idx += 2;
                if (idx >= cap) idx -= cap;
                k = 2;
                ahead = c.P[lb + (idx == 0 ? cap - 1 : idx - 1)];
            }
        }
        const float x = c.P[lb + idx];
        if (obs && (kSkip || k >= kMin)) {  // bin end: vehicles past the midpoint, position sum (time t)
            past += x >= __fmul_rn(g.x, 0.5f) ? 1 : 0;
            psum += pos_fx(x);
        }
        if (!kObsOnly && (kSkip || k >= kMin)) {
            const float h = (!kSkip && k == 0) ? M : __fsub_rn(ahead, x);
            int tag;
            c.P[lb + idx] = newell(x, h, g.x, g.y, g.z, g.w, tag);
            if (kTape) {                    // tape: branch tag of the slot, time-t position at bin ends
                const size_t o = (size_t)r * a.S + c.base0 + lb + idx;
                if (obs) d.tape_pos[o] = x;
                d.tag_tape[o] = (int8_t)tag;
            }
        }
        ahead = x;
        ++k;
        if (++idx == cap) idx = 0;
    }
    if (obs && v0 < v1) {
        atomicAdd(&S.past[li], past);
        atomicAdd(&S.psum[li], (unsigned long long)psum);
    }
}

// Observation at bin ends, choice, merge and records of this thread's link or
// origin queue.
template <bool kTape>
__device__ __forceinline__ void p_decide(const DevSim &d, const PArgs &a, PSmem &S, const PCtx &c, int t, bool obs,
                                         bool obs_only) {
    const int tid = threadIdx.x;
    unsigned long long *Wt = a.W3 + (size_t)(t % 3) * d.L;
    if (tid < c.nl) {
        const int li = tid, j = c.j0 + li;
        const int4 q = S.q[li];
        const int n = q.y;
        int4 stat = S.stat[li];
        if (obs) {
            const int bin = (t - 1) / d.obs_every;
            const size_t o = (size_t)bin * d.L + j;
            const int C = q.w + S.past[li];
            d.out_counts[o] = C - stat.w;
            const longlong2 ps = S.lpos[li];
            const long long pnow = (long long)S.psum[li];
            const long long dist = pnow - ps.x + ps.y;
            d.out_speed[o] = stat.x ? (float)((double)dist / (double)kPosScale / ((double)stat.x * (double)d.dt)) : 0.0f;
            d.out_tt[o] = stat.z ? (float)((double)stat.y * (double)d.dt / (double)stat.z) : 0.0f;
            stat = make_int4(0, 0, 0, C);
            S.lpos[li] = make_longlong2(pnow, 0);
            if (obs_only) { S.stat[li] = stat; return; }
        }
        stat.x += n;
        S.stat[li] = stat;
        const int4 c0 = S.cr[li];
        const int4 nd = S.nd[li];
        const int4 ld = S.ld[li];
        int tgt = kTgtNone;
        if (c0.x >= 0) {
            if (nd.y == ld.y) {
                tgt = kTgtSink;
            } else {
                tgt = p_choose(d, S, li, c.LO + nd.z, nd.w, ld.y, ld.x, t);
                red_max_u64(Wt + tgt, p_word(S.mkey[li], ld.x, ld.y, a.packz));
                if (kTape) d.tape_mkey[(size_t)(t - a.t0) * (d.L + d.V) + c.j0 + li] = S.mkey[li];
            }
        }
        const int4 st = S.st[li];
        const int lb = st.x - c.base0;
        auto at = [&](int k) {
            int idx = q.x + k;
            if (idx >= st.y) idx -= st.y;
            return c.P[lb + idx];
        };
        const float x0 = n >= 1 ? at(0) : 0.0f;
        const float xt = n >= 1 ? at(n - 1) : 0.0f;
        S.xt[li] = xt;                      // ahead of the next entrant (p_ends_pre)
        S.past[li] = 0;                     // the sums of the next step start from zero
        S.psum[li] = 0ull;
        // the record of step t (the transfers of step t add the next-step bits
        // of p_bits and set its final target)
        S.cr[li] = make_int4(c0.x, c0.x >= 0 ? tgt : kTgtNone, c0.z << 8, __float_as_int(x0));
    } else if (!obs_only && tid >= kPNodeTid && tid < kPNodeTid + c.nn) {
        const int ni = tid - kPNodeTid;
        const int2 r = S.nrec[ni];
        if (r.x < 0) return;
        const int4 nh = S.nh[ni];
        int tgt;
        if (S.nzone[ni] == nh.y) {
            tgt = kTgtSink;
        } else {
            const int4 nq = S.nq[ni];
            tgt = p_choose(d, S, kPLinks + ni, c.NO + nq.z, nq.w, nh.y, nh.x, t);
            red_max_u64(Wt + tgt, p_word(S.mkey[kPLinks + ni], nh.x, nh.y, a.packz));
            if (kTape) d.tape_mkey[(size_t)(t - a.t0) * (d.L + d.V) + d.L + c.n0 + ni] = S.mkey[kPLinks + ni];
        }
        S.nrec[ni] = make_int2(r.x, tgt);
    }
}

// Next-step vacancy and arrival bits of link li = threadIdx.x - kPBitsTid for
// the four (pop, push) outcomes of the coming transfers, from the positions
// after the step's car-following at queue positions 0, 1, n - 1 and n - 2: a
// vehicle entering at 0 finds the link vacant after the next car-following
// (rearmost vehicle beyond the jam spacing, SI-B) / the leader reaches the
// arrival line (Alg. S2).  Run beside the decisions by warps that hold no link
// or origin queue; the transfers of the next step add them to the record.
__device__ __forceinline__ void p_bits(const DevSim &d, PSmem &S, const PCtx &c) {
    const int li = threadIdx.x - kPBitsTid;
    if (li < 0 || li >= c.nl) return;
    const float M = d.M;
    const int4 q = S.q[li];
    const int n = q.y;
    const int4 st = S.st[li];
    const float4 g = S.g[li];
    const int lb = st.x - c.base0;
    auto at = [&](int k) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        return c.P[lb + idx];
    };
    const float4 x = make_float4(n >= 1 ? at(0) : 0.0f, n >= 2 ? at(1) : 0.0f,      // x0, x1,
                                 n >= 1 ? at(n - 1) : 0.0f, n >= 2 ? at(n - 2) : 0.0f);  // xt (rearmost), xpt
    int bits = 0;
    bits |= (n == 0 || vacant_after(x.z, n >= 2 ? __fsub_rn(x.w, x.z) : M, g)) << 0;
    bits |= (n <= 1 || vacant_after(x.z, n >= 3 ? __fsub_rn(x.w, x.z) : M, g)) << 1;
    bits |= vacant_after(0.0f, n >= 1 ? x.z : M, g) << 2;
    bits |= vacant_after(0.0f, n >= 2 ? x.z : M, g) << 3;
    bits |= (n >= 1 && arrives_after(x.x, g, M, d.eps_arr)) << 4;
    bits |= (n >= 2 && arrives_after(x.y, g, M, d.eps_arr)) << 5;
    bits |= arrives_after(n >= 1 ? x.x : 0.0f, g, M, d.eps_arr) << 6;
    bits |= arrives_after(n >= 2 ? x.y : 0.0f, g, M, d.eps_arr) << 7;
    S.nbits[li] = bits;
}

// First link of each car-following run of the barrier wait (p_carfollow with
// kMin = 2): run ct starts at vehicle v0 = floor(ct nv / kPCF), and v0 >= a
// exactly when ct >= ceil(a kPCF / nv), so link li (vehicles voff[li] ..
// voff[li+1] - 1) holds the first vehicle of runs ceil(voff[li] kPCF / nv) ..
// ceil(voff[li+1] kPCF / nv) - 1.  Runs without vehicles are not listed (nor
// read).  Written beside the decisions by the threads of p_bits.
__device__ __forceinline__ void p_run_links(PSmem &S, const PCtx &c) {
    const int li = threadIdx.x - kPBitsTid;
    if (li < 0 || li >= c.nl) return;
    const int nv = S.voff[c.nl];                             // < 2^16: a kPCF fits in 32 bits
    const int a = S.voff[li], b = S.voff[li + 1];
    if (a == b) return;
    const int lo = (a * kPCF + nv - 1) / nv, hi = (b * kPCF + nv - 1) / nv;
    for (int ct = lo; ct < hi; ++ct) S.cfli[ct] = li;
}

// tape: vehicle of every occupied slot at the start of the segment (record r =
// 0), by every warp once the choice and car-following work of its first step
// is done (the decisions that follow do not depend on it).  Later steps need no
// copy: the vehicle at queue position k of link j is entrant (exits + k) of j,
// either one that was queued at the segment start or one of the entrant log.
// A warp takes kTVL consecutive links at a time and issues the loads of their
// first 32 queue positions before any store, so that the L2 round trips
// overlap.
constexpr int kTVL = 4;

__device__ __forceinline__ void p_tape_vid(const DevSim &d, const PArgs &a, const PSmem &S, const PCtx &c, int r) {
    const int w = threadIdx.x >> 5, nw = kPT / 32, lane = threadIdx.x & 31;
    int *tv = d.tape_vid + (size_t)r * a.S;
    for (int l0 = w * kTVL; l0 < c.nl; l0 += nw * kTVL) {
        int gs[kTVL], v[kTVL];
#pragma unroll
        for (int j = 0; j < kTVL; ++j) {
            const int li = l0 + j;
            gs[j] = -1;
            if (li < c.nl) {
                const int2 qv = *reinterpret_cast<const int2 *>(&S.q[li]);
                if (lane < qv.y) {
                    const int lb = S.lbase[li], cap = S.lbase[li + 1] - lb;
                    int idx = qv.x + lane;
                    if (idx >= cap) idx -= cap;
                    gs[j] = c.base0 + lb + idx;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kTVL; ++j) v[j] = gs[j] >= 0 ? __ldcg(&d.saux[gs[j]].x) : 0;
#pragma unroll
        for (int j = 0; j < kTVL; ++j)
            if (gs[j] >= 0) tv[gs[j]] = v[j];
        for (int j = 0; j < kTVL; ++j) {            // queue positions 32, 64, ... of long queues, kTVL rounds at once
            const int li = l0 + j;
            if (li >= c.nl) break;
            const int2 qv = *reinterpret_cast<const int2 *>(&S.q[li]);
            const int lb = S.lbase[li], cap = S.lbase[li + 1] - lb;
            for (int k0 = 32; k0 < qv.y; k0 += 32 * kTVL) {
#pragma unroll
                for (int m = 0; m < kTVL; ++m) {
                    const int k = k0 + 32 * m + lane;
                    gs[m] = -1;
                    if (k < qv.y) {
                        int idx = qv.x + k;
                        if (idx >= cap) idx -= cap;
                        gs[m] = c.base0 + lb + idx;
                    }
                }
#pragma unroll
                for (int m = 0; m < kTVL; ++m) v[m] = gs[m] >= 0 ? __ldcg(&d.saux[gs[m]].x) : 0;
#pragma unroll
                for (int m = 0; m < kTVL; ++m)
                    if (gs[m] >= 0) tv[gs[m]] = v[m];
            }
        }
    }
}

template <bool kTape>
__device__ __forceinline__ void persist_body(const DevSim &d, const PArgs &a) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PSmem &S = *reinterpret_cast<PSmem *>(p_smem);
    const int tid = threadIdx.x;
    PCtx c;
    c.j0 = a.grp_links[blockIdx.x];
    c.nl = a.grp_links[blockIdx.x + 1] - c.j0;
    c.n0 = blockIdx.x * a.npg;
    c.nn = max(0, min(a.npg, d.V - c.n0));
    c.base0 = c.nl > 0 ? d.lst[c.j0].x : 0;
    const int nslots = c.nl > 0 ? d.lst[c.j0 + c.nl - 1].x + d.lst[c.j0 + c.nl - 1].y - c.base0 : 0;
    c.nslots = nslots;
    c.lo0 = c.nl > 0 ? d.lnode[c.j0].z : 0;
    const int n_lo = c.nl > 0 ? d.lnode[c.j0 + c.nl - 1].w - c.lo0 : 0;
    c.no0 = c.nn > 0 ? d.no_ptr[c.n0] : 0;
    const int n_no = c.nn > 0 ? d.no_ptr[c.n0 + c.nn] - c.no0 : 0;
    unsigned char *dyn = p_smem + sizeof(PSmem);
    c.P = reinterpret_cast<float *>(dyn);
    float4 *LO = reinterpret_cast<float4 *>(dyn + p_dyn_bytes(nslots, 0, 0));
    float4 *NO = LO + n_lo;
    c.LO = LO;
    c.NO = NO;
    // ---------------- load the group's state ----------------
    const float *pc = (a.t0 & 1) ? d.pos1 : d.pos0;
    for (int s = tid; s < nslots; s += kPT) c.P[s] = pc[c.base0 + s];
    for (int e = tid; e < n_lo; e += kPT) LO[e] = d.loinfo[c.lo0 + e];
    for (int e = tid; e < n_no; e += kPT) NO[e] = d.noinfo[c.no0 + e];
    for (int li = tid; li < c.nl; li += kPT) {
        const int j = c.j0 + li;
        const int4 q = d.lq[j], st = d.lst[j], nd = d.lnode[j];
        S.q[li] = q;
        S.st[li] = st;
        S.lbase[li] = st.x - c.base0;
        S.g[li] = d.geo[j];
        S.nd[li] = make_int4(nd.x, nd.y, nd.z - c.lo0, nd.w - nd.z);
        S.stat[li] = d.lstat[j];
        S.past[li] = 0;
        S.psum[li] = 0ull;
        S.lpos[li] = d.lpos[j];
        S.flags[li] = d.vac[j];
        if (!(d.vac[j] & kFlagVacant))                     // read by the transfers of step t0
            a.W3[(size_t)(a.t0 % 3) * d.L + j] = kWBlocked;
        S.cr[li] = d.crec[j];
        S.alpha[li] = d.alpha[j];
        int4 ld = make_int4(-1, -1, -1, -1);
        int2 le = make_int2(0, 0);
        if (q.y >= 1) {
            const int2 v = d.saux[st.x + q.x];
            ld.x = v.x;
            ld.y = v.y;
            le.x = d.sentry[st.x + q.x];
        }
        if (q.y >= 2) {
            const int idx = q.x + 1 >= st.y ? q.x + 1 - st.y : q.x + 1;
            const int2 v = d.saux[st.x + idx];
            ld.z = v.x;
            ld.w = v.y;
            le.y = d.sentry[st.x + idx];
        }
        S.ld[li] = ld;
        S.le[li] = le;
    }
    for (int ni = tid; ni < c.nn; ni += kPT) {
        const int n = c.n0 + ni;
        const int ptr = d.fifo_ptr[n], end = d.fifo_end[n];
        const int o0 = d.no_ptr[n], o1 = d.no_ptr[n + 1];
        S.nq[ni] = make_int4(ptr, end, o0 - c.no0, o1 - o0);
        S.nzone[ni] = d.node_zone[n];
        S.nrec[ni] = d.nrec[n];
        int4 nh = make_int4(-1, -1, -1, -1);
        int2 dp = make_int2(0, 0);
        if (ptr < end) {
            const int2 v = d.fifo_list[ptr];
            nh.x = v.x;
            nh.y = v.y;
            dp.x = d.fifo_dep[ptr];
        }
        if (ptr + 1 < end) {
            const int2 v = d.fifo_list[ptr + 1];
            nh.z = v.x;
            nh.w = v.y;
            dp.y = d.fifo_dep[ptr + 1];
        }
        S.nh[ni] = nh;
        S.ndep[ni] = dp;
    }
    if (tid < 4) S.cnt[tid] = 0;
    if (tid == 0) {
        S.stop = 0;
        S.lbase[c.nl] = nslots;
    }
    __syncthreads();
    // ---------------- steps ----------------
    // Step t: its car-following runs in two parts.  The vehicles at queue
    // positions >= 2 of the queues as step t - 1 leaves them do not depend on
    // the transfers of t - 1 (their vehicle ahead stays), so they are updated
    // while the CTA waits at the grid barrier of step t - 1; the first two and
    // the entrant follow in the transfers (p_ends_pre, p_ends_post).  The first step of the
    // launch, with no transfers pending, updates every vehicle before its
    // choices.
    unsigned epoch = 0;
    for (int t = a.t0; t < a.t1; ++t) {
        const bool first = t == a.t0;
        const bool obs = t > 0 && t % d.obs_every == 0;
        PPend pd{};
        int cnt[4] = {0, 0, 0, 0};
        if (!first) p_apply<kTape>(d, a, S, c, t - 1, pd, cnt, true, obs);
        // reads what this thread's p_apply wrote; the offsets of the scan count
        // the vehicles the step's car-following runs take: all of them on the
        // first step, else those at queue positions >= 2 when the launch runs
        // over those only (skip2: long queues; with short ones the runs would
        // step over many links that hold no such vehicle)
        const int v = p_candidate<kTape>(d, S, c, t, t - a.t0, false, first || !a.skip2);
        if (!first) p_count_bal(S, cnt);
        p_scan(S, c, v);
        if (first) {
            p_carfollow<kTape, false, 0>(d, a, S, c, t - a.t0, obs);
            __syncthreads();
        }
        p_pairs(d, a, S, c, t);
        if (!first && (tid >> 5) == kPT / 32 - 1) p_count_sum(d, S, t - 1);   // the last warp rarely holds pairs
        __syncthreads();
        if (kTape && t == a.t0) p_tape_vid(d, a, S, c, 0);     // vehicles of the segment start
        p_decide<kTape>(d, a, S, c, t, obs, false);
        p_bits(d, S, c);
        p_run_links(S, c);
        p_refill(S, c, pd);
        ++epoch;
        grid_arrive(a.bar);
        if (t + 1 < a.t1) {
            const bool obs1 = (t + 1) % d.obs_every == 0;
            if (first || !a.skip2) p_carfollow<kTape, false, 2>(d, a, S, c, t + 1 - a.t0, obs1);
            else p_carfollow<kTape, false, 2, true>(d, a, S, c, t + 1 - a.t0, obs1);
        }
        if (!grid_wait(d, a.bar, epoch * gridDim.x + (unsigned)a.bar_extra, t, &S.stop)) return;
    }
    if (a.t1 > a.t0) {
        PPend pd{};
        int cnt[4] = {0, 0, 0, 0};
        p_apply<kTape>(d, a, S, c, a.t1 - 1, pd, cnt, false, false);
        p_count(S, cnt);
        p_refill(S, c, pd);
        __syncthreads();
        if (tid < 4 && S.cnt[tid]) atomicAdd(&d.step_delta[4 * (a.t1 - 1) + tid], S.cnt[tid]);
    }
    if (a.final_obs) {
        __syncthreads();
        const int v = p_candidate<false>(d, S, c, a.t1, 0, true);
        p_scan(S, c, v);
        p_carfollow<false, true, 0>(d, a, S, c, 0, true);
        __syncthreads();
        p_decide<false>(d, a, S, c, a.t1, true, true);
    }
    __syncthreads();
    // ---------------- write the group's state back ----------------
    // merge words as the two-kernel executor leaves them: those of the last
    // step (standard format) in its parity buffer, the other buffer zero
    float *pdst = (a.t1 & 1) ? d.pos1 : d.pos0;
    for (int s = tid; s < nslots; s += kPT) pdst[c.base0 + s] = c.P[s];
    const unsigned long long *Wl = a.W3 + (size_t)((a.t1 + 2) % 3) * d.L;
    unsigned long long *Wlast = (a.t1 & 1) ? d.W0 : d.W1;
    unsigned long long *Wnext = (a.t1 & 1) ? d.W1 : d.W0;
    for (int li = tid; li < c.nl; li += kPT) {
        const int j = c.j0 + li;
        d.lq[j] = S.q[li];
        d.lstat[j] = S.stat[li];
        d.lpos[j] = S.lpos[li];
        d.vac[j] = S.flags[li];
        d.crec[j] = S.cr[li];
        if (a.t1 > a.t0) {          // a word on a link that was not vacant names no entrant
            unsigned long long w = __ldcg(Wl + j);
            if (w == kWBlocked) w = 0ull;
            Wlast[j] = w ? ((w & 0xffffffff00000000ull) | (unsigned long long)(~(uint32_t)p_vid(w, a.packz))) : 0ull;
        }
        Wnext[j] = 0ull;
    }
    for (int ni = tid; ni < c.nn; ni += kPT) {
        const int n = c.n0 + ni;
        d.fifo_ptr[n] = S.nq[ni].x;
        d.nrec[n] = S.nrec[ni];
    }
}

__global__ void __launch_bounds__(kPT, 1) k_persist(DevSim d, PArgs a) { persist_body<false>(d, a); }

// the same run recording the reverse pass's tape (d.tape_* and d.tag_tape are
// the bases of record 0 = step a.t0; slot records have stride a.S)
__global__ void __launch_bounds__(kPT, 1) k_persist_tape(DevSim d, PArgs a) { persist_body<true>(d, a); }

}  // namespace ts
