// Step kernels of one simulator instance (sm_103a).
//
// One step phi = g o f runs as two kernels.
//
// k_step_a -- link blocks and origin-node blocks.
//   A link block owns a contiguous set of links whose queue capacities add up to
//   at most the block's shared-memory stage (links are packed on the host; a link
//   larger than the stage gets a block of its own).  Four phases separated by
//   barriers, each issuing one round of independent global loads:
//   P1  one thread per link: queue state, link data, statistics and flags of the
//       step; outflow credit; candidate = leader flagged as arriving with credit.
//   P2  all threads: every queue position of the block's links into shared
//       memory (kU coalesced loads in flight per thread whatever the queue
//       lengths); the leader's (vehicle, zone, entry step) and the choice-set
//       records of candidates.
//   P3  all threads: Newell car-following of every vehicle (SI-A, Eq.
//       newell_model) from the staged time-t positions into the other position
//       buffer; the utility + Gumbel key of every staged choice slot (SI-B Eqs.
//       softmax, gumbel, straigththrough) with the destination feature and the
//       vacancy of the slot's link; the merge key alpha + g' of each candidate.
//       At observation steps also the per-link midpoint count and position sum
//       (one segmented warp reduction per 32 staged elements).
//   P4  one thread per link: observation output when a bin closes (SI-D); argmax
//       over the slots (ties to the lowest slot) and the merge (SI-B "Merge
//       choice") as a 64-bit atomicMax of (alpha + g', ~vehicle id) into the
//       target's word; the vacancy X_min > dn/kappa and leader-arrival flags of
//       the next step for each of the four (pop, push) outcomes of this step.
//   Origin-node blocks: one thread per node handles the head of its origin queue
//   (a virtual inflow link of length 0) the same way.
// k_step_b -- one thread per link / origin node: applies the transfers (SI-B Eq.
//   transfer): pops the leader that won its merge or left to its destination,
//   pushes the merge winner at x = 0, updates credit, exits and link times, and
//   selects the next step's vacancy / arrival flags.
//
// Mean speed of a bin needs the distance sum sum_t sum_i (x_i(t+1) - x_i(t)) over
// the link's vehicles.  It telescopes: with P(t) the sum of the positions on the
// link at time t, the bin's distance is P(end) - P(start) + the post-f positions
// of the vehicles that left during the bin, so positions are summed only when a
// bin closes (fixed point 2^-16 m, exact integer sums in any order).
#pragma once
#include "ts_sim.cuh"

namespace ts {

// flags of link j for the coming step: bit 0 vacant, bit 1 leader arrives
constexpr int kFlagVacant = 1, kFlagArrive = 2;
constexpr int kLinksPerBlock = 64;     // at most this many links per block
constexpr int kNodesPerBlock = 32;     // at most this many origin queues per block
constexpr int kMaxSlotsStaged = 4;     // choice slots per link evaluated in P3
constexpr int kBlockA = 256;           // threads of k_step_a
constexpr int kU = 8;                  // staged elements per thread per pass
constexpr float kPosScale = 65536.0f;  // position sums: fixed point 2^-16 m

__device__ __forceinline__ bool vacant_after(float x, float h, float4 g) {
    int tag;
    return newell(x, h, g.x, g.y, g.z, g.w, tag) > g.z;
}
__device__ __forceinline__ bool arrives_after(float x, float4 g, float M, float eps) {
    int tag;
    return newell(x, M, g.x, g.y, g.z, g.w, tag) >= __fsub_rn(g.x, eps);
}
__device__ __forceinline__ long long pos_fx(float x) { return __float2ll_rn(__fmul_rn(x, kPosScale)); }

struct ABlockSmem {
    int4 q[kLinksPerBlock];             // queue head, length, credit, exits
    int4 st[kLinksPerBlock];            // queue base, capacity, q_fx, credit cap
    float4 g[kLinksPerBlock];           // length, u dt, s, tag band
    int4 nd[kLinksPerBlock];            // head node, head zone, choice begin/end
    int4 stat[kLinksPerBlock];          // vehicle-steps, link-time sum, leavers, C_prev
    longlong2 ps[kLinksPerBlock];       // position sum at bin start, leavers' positions
    int off[kLinksPerBlock + 1];        // first staged element of each link
    int cand[kLinksPerBlock];           // 1 candidate, 0 none
    int credit[kLinksPerBlock];
    float alpha[kLinksPerBlock];
    int2 lead[kLinksPerBlock];          // candidate (vehicle, zone)
    int ent[kLinksPerBlock];            // candidate entry step
    float mkey[kLinksPerBlock];         // candidate merge key alpha + g'
    int past[kLinksPerBlock];           // vehicles past the midpoint (observation)
    unsigned long long psum[kLinksPerBlock];  // position sum (observation)
    float4 x4[kLinksPerBlock];          // new positions of vehicles 0, 1, n-2, n-1
    float4 lo[kLinksPerBlock][kMaxSlotsStaged];
    float key[kLinksPerBlock][kMaxSlotsStaged];
    int vacm[kLinksPerBlock][kMaxSlotsStaged];
    // origin queues of the block's nodes
    int4 nq[kNodesPerBlock];            // next vehicle, end of queue, out-links begin/end
    int2 nlead[kNodesPerBlock];         // head (vehicle, zone); vehicle -1 if none departed
    int nzone[kNodesPerBlock];          // zone of the node
    float nmkey[kNodesPerBlock];
    float4 nlo[kNodesPerBlock][kMaxSlotsStaged];
    float nkey[kNodesPerBlock][kMaxSlotsStaged];
    int nvacm[kNodesPerBlock][kMaxSlotsStaged];
};

// element e of the block's staged queues -> local link index (binary search)
__device__ __forceinline__ int link_of(const int *off, int nl, int e) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// advance link index li (the link of an earlier element) to the link of
// element e: two linear steps, then a binary search (empty links have equal
// offsets, so the link of a later element can be many links further on)
__device__ __forceinline__ int link_advance(const int *off, int nl, int li, int e) {
    if (off[li + 1] > e) return li;
    ++li;
    if (off[li + 1] > e) return li;
    ++li;
    if (off[li + 1] > e) return li;
    return link_of(off, nl, e);
}

__device__ __forceinline__ float choice_key(const DevSim &d, float4 e, int zone, int vid, int t, int slot) {
    const float df = d.dest_feat[(size_t)zone * d.V + __float_as_int(e.z)];
    const float v = __fadd_rn(e.x, __fmul_rn(e.y, df));
    return __fadd_rn(v, gumbel(d.key0, d.key1, vid, t, 0, slot));
}

// Node-model choice of one candidate from its staged slots: argmax of the keys
// (ties to the lowest slot), slots past the stage evaluated inline.  Returns the
// target link, or kTgtBlocked when the chosen link is not vacant.
__device__ __forceinline__ int choose(const DevSim &d, const float4 *lo, const float *key, const int *vacm,
                                      const float4 *info, int deg, int zone, int vid, int t) {
    float bk = -INFINITY;
    int bm = -1, bv = 0;
    for (int k = 0; k < deg; ++k) {
        float kk;
        int m, vm;
        if (k < kMaxSlotsStaged) {
            kk = key[k];
            m = __float_as_int(lo[k].w);
            vm = vacm[k];
        } else {
            const float4 e = info[k];
            kk = choice_key(d, e, zone, vid, t, k);
            m = __float_as_int(e.w);
            vm = d.vac[m] & kFlagVacant;
        }
        if (bm < 0 || kk > bk) { bk = kk; bm = m; bv = vm; }
    }
    return bv ? bm : kTgtBlocked;
}

// One block of k_step_a: links [blk_links[b], blk_links[b+1]) and origin queues
// [b npb, (b+1) npb), phase by phase (see the file header).  kTape: also write
// the reverse pass's tape of the step (state at its start for the occupied
// slots, tags, queue states and records).
template <bool kTape>
__device__ __forceinline__ void step_block(const DevSim &d, int b, int t, bool obs_only, float *xs) {
    __shared__ ABlockSmem S;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int j0 = d.blk_links[b];
    const int nl = d.blk_links[b + 1] - j0;
    const int n0 = b * d.npb;
    const int nn = obs_only ? 0 : max(0, min(d.npb, d.V - n0));
    const int ni = tid - kLinksPerBlock;             // origin-queue index of this thread
    const int p = t & 1;
    const float *pc = p ? d.pos1 : d.pos0;
    float *pn = p ? d.pos0 : d.pos1;
    const bool obs = obs_only || (t > 0 && t % d.obs_every == 0);
    // ---------------- P1: link data, statistics, credit, candidate; queue pointers ----------------
    if (tid < nl) {
        const int j = j0 + tid;
        const int4 q = d.lq[j];
        const int4 st = d.lst[j];
        const int flags = d.vac[j];
        if (kTape) d.tape_lq[j] = q;
        S.q[tid] = q;
        S.st[tid] = st;
        if (q.y > 0 || obs) {              // an empty link off a bin end needs only its credit
            S.g[tid] = d.geo[j];
            S.nd[tid] = d.lnode[j];
            S.stat[tid] = d.lstat[j];
            S.ps[tid] = d.lpos[j];
            S.alpha[tid] = d.alpha[j];
        }
        const int credit = min(q.z + st.z, st.w);
        S.credit[tid] = credit;
        S.cand[tid] = !obs_only && q.y > 0 && (flags & kFlagArrive) && credit >= d.dn_fx;
        S.past[tid] = 0;
        S.psum[tid] = 0ull;
        S.ent[tid] = 0;
        S.lead[tid] = make_int2(-1, -1);
    } else if (ni >= 0 && ni < nn) {
        const int n = n0 + ni;
        S.nq[ni] = make_int4(d.fifo_ptr[n], d.fifo_end[n], d.no_ptr[n], d.no_ptr[n + 1]);
        S.nzone[ni] = d.node_zone[n];
        S.nlead[ni] = make_int2(-1, -1);
    }
    __syncthreads();
    if (tid < 32) {          // exclusive scan of queue lengths (nl <= 64)
        const int a = tid < nl ? S.q[tid].y : 0;
        const int c = tid + 32 < nl ? S.q[tid + 32].y : 0;
        int sa = a, sc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(kFull, sa, o), yc = __shfl_up_sync(kFull, sc, o);
            if (tid >= o) { sa += ya; sc += yc; }
        }
        const int tot_a = __shfl_sync(kFull, sa, 31);
        if (tid < nl) S.off[tid] = sa - a;
        if (tid + 32 < nl) S.off[tid + 32] = tot_a + sc - c;
        if (tid == 31) S.off[nl] = tot_a + sc;
    }
    __syncthreads();
    const int total = S.off[nl];
    // ---------------- P2: stage positions, leaders, queue heads and choice records ----------------
    // Warp w stages elements [pass + 32 kU w, pass + 32 kU (w + 1)); the link of
    // an element is tracked linearly from a binary search on the first one.
    for (int pass = 0; pass < total; pass += kBlockA * kU) {
        const int wbase = pass + (tid >> 5) * 32 * kU;
        if (wbase >= total) break;
        int li = link_of(S.off, nl, min(wbase + lane, total - 1));
        float v[kU];
        int sl[kTape ? kU : 1], vd[kTape ? kU : 1];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = wbase + u * 32 + lane;
            v[u] = 0.0f;
            if (e < total) {
                li = link_advance(S.off, nl, li, e);
                const int4 q = S.q[li], st = S.st[li];
                int idx = q.x + (e - S.off[li]);
                if (idx >= st.y) idx -= st.y;
                v[u] = pc[st.x + idx];
                if (kTape) {
                    sl[u] = st.x + idx;
                    if (d.tape_vid) vd[u] = d.saux[st.x + idx].x;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = wbase + u * 32 + lane;
            if (e < total) {
                xs[e] = v[u];
                if (kTape) {
                    if (obs) d.tape_pos[sl[u]] = v[u];           // read only at bin ends
                    if (d.tape_vid) d.tape_vid[sl[u]] = vd[u];
                }
            }
        }
    }
    if (tid < nl && S.cand[tid]) {
        const int4 q = S.q[tid], st = S.st[tid];
        S.lead[tid] = d.saux[st.x + q.x];
        S.ent[tid] = d.sentry[st.x + q.x];
    } else if (ni >= 0 && ni < nn) {
        const int4 nq = S.nq[ni];
        if (nq.x < nq.y) {                       // both loads issued before the test
            const int dep = d.fifo_dep[nq.x];
            const int2 head = d.fifo_list[nq.x];
            if (dep <= t) S.nlead[ni] = head;
        }
    }
    if (!obs_only) {
        for (int c = tid; c < (kLinksPerBlock + kNodesPerBlock) * kMaxSlotsStaged; c += kBlockA) {
            const int r = c / kMaxSlotsStaged, k = c % kMaxSlotsStaged;
            if (r < kLinksPerBlock) {
                if (r >= nl) continue;
                const int4 nd = S.nd[r];
                if (S.cand[r] && k < nd.w - nd.z) S.lo[r][k] = d.loinfo[nd.z + k];
            } else {
                const int q = r - kLinksPerBlock;
                if (q >= nn) continue;
                const int4 nq = S.nq[q];          // queue not empty: stage speculatively
                if (nq.x < nq.y && k < nq.w - nq.z) S.nlo[q][k] = d.noinfo[nq.z + k];
            }
        }
    }
    __syncthreads();
    // ---------------- P3: car-following, choice and merge keys ----------------
    if (!obs_only) {
        for (int c = tid; c < (kLinksPerBlock + kNodesPerBlock) * kMaxSlotsStaged; c += kBlockA) {
            const int r = c / kMaxSlotsStaged, k = c % kMaxSlotsStaged;
            if (r < kLinksPerBlock) {
                if (r >= nl || !S.cand[r]) continue;
                const int4 nd = S.nd[r];
                const int2 lead = S.lead[r];
                if (k == 0) S.mkey[r] = __fadd_rn(S.alpha[r], gumbel(d.key0, d.key1, lead.x, t, 1, 0));
                if (k >= nd.w - nd.z || nd.y == lead.y) continue;   // no slot / leaves to its destination
                const float4 e = S.lo[r][k];
                S.key[r][k] = choice_key(d, e, lead.y, lead.x, t, k);
                S.vacm[r][k] = d.vac[__float_as_int(e.w)] & kFlagVacant;
            } else {
                const int q = r - kLinksPerBlock;
                if (q >= nn) continue;
                const int2 lead = S.nlead[q];
                if (lead.x < 0) continue;
                const int4 nq = S.nq[q];
                if (k == 0) S.nmkey[q] = __fadd_rn(d.alpha[d.L], gumbel(d.key0, d.key1, lead.x, t, 1, 0));
                if (k >= nq.w - nq.z || S.nzone[q] == lead.y) continue;
                const float4 e = S.nlo[q][k];
                S.nkey[q][k] = choice_key(d, e, lead.y, lead.x, t, k);
                S.nvacm[q][k] = d.vac[__float_as_int(e.w)] & kFlagVacant;
            }
        }
    }
    for (int pass = 0; pass < total; pass += kBlockA * kU) {
        const int wbase = pass + (tid >> 5) * 32 * kU;
        if (wbase >= total) break;
        int li = link_of(S.off, nl, min(wbase + lane, total - 1));
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = wbase + u * 32 + lane;
            const bool act = e < total;
            float x = 0.0f;
            if (act) {
                li = link_advance(S.off, nl, li, e);
                x = xs[e];
                if (!obs_only) {
                    const int k = e - S.off[li];
                    const int4 q = S.q[li], st = S.st[li];
                    const float4 g = S.g[li];
                    const float h = (k == 0) ? d.M : __fsub_rn(xs[e - 1], x);
                    int tag;
                    const float xn = newell(x, h, g.x, g.y, g.z, g.w, tag);
                    int idx = q.x + k;
                    if (idx >= st.y) idx -= st.y;
                    pn[st.x + idx] = xn;
                    if (kTape) d.tag_tape[st.x + idx] = (int8_t)tag;
                    // keep the new positions of the first two and last two vehicles
                    if (k == 0) S.x4[li].x = xn;
                    if (k == 1) S.x4[li].y = xn;
                    if (k == q.y - 2) S.x4[li].z = xn;
                    if (k == q.y - 1) S.x4[li].w = xn;
                }
            }
            if (obs) {      // block-uniform: midpoint count and position sum per link
                const unsigned seg = __match_any_sync(kFull, act ? li : -1);
                const unsigned past = act && x >= __fmul_rn(S.g[li].x, 0.5f) ? 1u : 0u;
                const unsigned sp = __reduce_add_sync(seg, past);
                // exact 64-bit segment sum from two 32-bit reductions of
                // 24-bit pieces (no carry is lost for positions below 2^31 m)
                const long long xf = act ? pos_fx(x) : 0;
                const unsigned slo = __reduce_add_sync(seg, (unsigned)(xf & 0xffffffll));
                const unsigned shi = __reduce_add_sync(seg, (unsigned)(xf >> 24));
                if (act && lane == __ffs(seg) - 1) {
                    if (sp) atomicAdd(&S.past[li], (int)sp);
                    atomicAdd(&S.psum[li], (unsigned long long)slo + ((unsigned long long)shi << 24));
                }
            }
        }
    }
    __syncthreads();
    // ---------------- P4: observation, choice, merge, next-step flags ----------------
    if (ni >= 0 && ni < nn) {            // origin queue heads
        const int n = n0 + ni;
        const int2 lead = S.nlead[ni];
        int tgt = kTgtNone;
        if (lead.x >= 0) {
            if (S.nzone[ni] == lead.y) {
                tgt = kTgtSink;
            } else {
                const int4 nq = S.nq[ni];
                tgt = choose(d, S.nlo[ni], S.nkey[ni], S.nvacm[ni], d.noinfo + nq.z, nq.w - nq.z, lead.y, lead.x, t);
                if (tgt >= 0) atomicMax(p ? &d.W1[tgt] : &d.W0[tgt], merge_word(S.nmkey[ni], lead.x));
                if (kTape && tgt >= 0) d.tape_mkey[d.L + n] = S.nmkey[ni];
            }
        }
        d.nrec[n] = make_int2(lead.x, tgt);
        if (kTape) d.tape_nrec[n] = make_int2(lead.x, tgt);
        return;
    }
    if (tid >= nl) return;
    const int li = tid, j = j0 + tid;
    const int4 q = S.q[li];
    const int n = q.y;
    if (n == 0 && !obs) {                  // empty link: credit, and the static bits of an empty queue
        d.lq[j].z = S.credit[li];
        const int4 rec = make_int4(-1, kTgtNone, d.ebits[j], 0);
        d.crec[j] = rec;
        if (kTape) d.tape_crec[j] = rec;
        return;
    }
    int4 stat = S.stat[li];
    longlong2 ps = S.ps[li];
    if (obs) {
        const int bin = (t - 1) / d.obs_every;
        const size_t o = (size_t)bin * d.L + j;
        const int C = q.w + S.past[li];
        d.out_counts[o] = C - stat.w;
        const long long pnow = (long long)S.psum[li];
        const long long dist = pnow - ps.x + ps.y;
        d.out_speed[o] = stat.x ? (float)((double)dist / (double)kPosScale / ((double)stat.x * (double)d.dt)) : 0.0f;
        d.out_tt[o] = stat.z ? (float)((double)stat.y * (double)d.dt / (double)stat.z) : 0.0f;
        stat = make_int4(0, 0, 0, C);
        ps = make_longlong2(pnow, 0);
        d.lpos[j] = ps;
        if (obs_only) { d.lstat[j] = stat; return; }
    }
    stat.x += n;
    d.lstat[j] = stat;
    const float4 g = S.g[li];
    const int4 nd = S.nd[li];
    int tgt = kTgtNone;
    const int2 lead = S.lead[li];
    if (S.cand[li]) {
        if (nd.y == lead.y) {
            tgt = kTgtSink;
        } else {
            tgt = choose(d, S.lo[li], S.key[li], S.vacm[li], d.loinfo + nd.z, nd.w - nd.z, lead.y, lead.x, t);
            if (tgt >= 0) atomicMax(p ? &d.W1[tgt] : &d.W0[tgt], merge_word(S.mkey[li], lead.x));
            if (kTape && tgt >= 0) d.tape_mkey[j] = S.mkey[li];
        }
    }
    d.lq[j].z = S.credit[li];
    // flags of the next step for each outcome o = pop | push << 1
    const float M = d.M;
    const float4 x4 = S.x4[li];
    const float x0 = n >= 1 ? x4.x : 0.0f;
    const float x1 = n >= 2 ? x4.y : 0.0f;
    const float xt = n >= 1 ? x4.w : 0.0f;
    const float xpt = n >= 2 ? x4.z : 0.0f;
    int bits = 0;
    bits |= (n == 0 || vacant_after(xt, n >= 2 ? __fsub_rn(xpt, xt) : M, g)) << 0;
    bits |= (n <= 1 || vacant_after(xt, n >= 3 ? __fsub_rn(xpt, xt) : M, g)) << 1;
    bits |= vacant_after(0.0f, n >= 1 ? xt : M, g) << 2;
    bits |= vacant_after(0.0f, n >= 2 ? xt : M, g) << 3;
    bits |= (n >= 1 && arrives_after(x0, g, M, d.eps_arr)) << 4;
    bits |= (n >= 2 && arrives_after(x1, g, M, d.eps_arr)) << 5;
    bits |= arrives_after(n >= 1 ? x0 : 0.0f, g, M, d.eps_arr) << 6;
    bits |= arrives_after(n >= 2 ? x1 : 0.0f, g, M, d.eps_arr) << 7;
    const int cand = S.cand[li];
    const int4 rec = make_int4(cand ? lead.x : -1, cand ? tgt : kTgtNone, (S.ent[li] << 8) | bits, __float_as_int(x0));
    d.crec[j] = rec;
    if (kTape) d.tape_crec[j] = rec;
}

__global__ void __launch_bounds__(kBlockA, 6) k_step_a(DevSim d, int t, int obs_only) {
    extern __shared__ float xs[];
    step_block<false>(d, blockIdx.x, t, obs_only != 0, xs);
}

// the same step, recording the reverse pass's tape (segment recomputation)
__global__ void __launch_bounds__(kBlockA, 6) k_step_a_tape(DevSim d, int t) {
    extern __shared__ float xs[];
    step_block<true>(d, blockIdx.x, t, false, xs);
}

// Sum of v over the block added to *dst by one atomic (every thread must call).
__device__ __forceinline__ void block_count(int v, int *dst, int *smem) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) smem[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < nw; ++k) s += smem[k];
        if (s) atomicAdd(dst, s);
    }
    __syncthreads();
}

// Transfers of step t for link / origin node i; adds this element's origin
// releases, arrivals, candidates and entries to c[0..3].
__device__ __forceinline__ void step_b_core(const DevSim &d, int i, int t, int c4[4]) {
    const int p = t & 1;
    const unsigned long long *W = p ? d.W1 : d.W0;
    int released = 0, arrived = 0, entered = 0, cands = 0;
    if (i < d.L) {
        const int j = i;
        float *pn = p ? d.pos0 : d.pos1;
        int4 q = d.lq[j];
        const int4 st = d.lst[j];
        const int4 c = d.crec[j];
        const unsigned long long win = W[j];
        if (d.tape_W) d.tape_W[j] = win;
        // second round, issued before any of it is used: the target's merge
        // word, the bin statistics a pop updates, the pushed vehicle's zone
        const bool push = win != 0ull;
        const int v = push ? merge_vid(win) : 0;
        unsigned long long wt = 0ull;
        int4 stat = make_int4(0, 0, 0, 0);
        longlong2 ps = make_longlong2(0, 0);
        int vz = 0;
        if (c.y >= 0) wt = W[c.y];
        if (c.x >= 0) {
            stat = d.lstat[j];
            ps = d.lpos[j];
        }
        int rl = 0;
        if (push) {
            vz = d.dest_zone[v];
            if (d.route_log) rl = d.route_len[v];
        }
        bool pop = false;
        cands = c.x >= 0;
        if (c.y == kTgtSink) {
            pop = true;
            d.vstate[c.x] = kVehArrived;
            arrived = 1;
        } else if (c.y >= 0) {
            pop = (wt != 0ull) && merge_vid(wt) == c.x;
        }
        if (pop) {
            stat.y += t + 1 - (c.z >> 8);
            stat.z += 1;
            ps.y += pos_fx(__int_as_float(c.w));
            d.lstat[j] = stat;
            d.lpos[j] = ps;
            q.x = (q.x + 1 == st.y) ? 0 : q.x + 1;
            q.y -= 1;
            q.z -= d.dn_fx;
            q.w += 1;
        }
        if (push) {
            if (q.y >= st.y) {
                set_error(d, SIM_EOVERFLOW, j, t);
            } else {
                int idx = q.x + q.y;
                if (idx >= st.y) idx -= st.y;
                pn[st.x + idx] = 0.0f;
                d.saux[st.x + idx] = make_int2(v, vz);
                d.sentry[st.x + idx] = t + 1;
                if (d.tape_ent) {                  // entrant log of the segment (reverse pass)
                    const int4 q0 = d.tape_lq0[j];
                    const int m = q.w + q.y - (q0.w + q0.y);
                    if (m >= 0 && m < d.tape_K) d.tape_ent[(size_t)j * d.tape_K + m] = v;
                    else set_error(d, SIM_EOVERFLOW, j, t);
                }
                q.y += 1;
                d.vstate[v] = j;
                entered = 1;
                if (d.route_log) {                 // route log for the reverse pass
                    const int r = rl;
                    if (r < d.route_cap) {
                        d.route_log[(size_t)v * d.route_cap + r] = make_int2(t, j);
                        d.route_len[v] = r + 1;
                    } else {
                        set_error(d, SIM_EOVERFLOW, -1 - v, t);
                    }
                }
            }
        }
        (p ? d.W0 : d.W1)[j] = 0ull;
        d.lq[j] = q;
        const int o = (pop ? 1 : 0) | (push ? 2 : 0);
        d.vac[j] = ((c.z >> o) & 1) | (((c.z >> (4 + o)) & 1) << 1);
    } else if (i < d.L + d.V) {
        const int n = i - d.L;
        const int2 c = d.nrec[n];
        cands = c.x >= 0;
        if (c.y == kTgtSink) {
            d.fifo_ptr[n] += 1;
            d.vstate[c.x] = kVehArrived;
            released = 1;
            arrived = 1;
        } else if (c.y >= 0) {
            const unsigned long long w = W[c.y];
            if (w != 0ull && merge_vid(w) == c.x) { d.fifo_ptr[n] += 1; released = 1; }
        }
    }
    c4[0] += released;
    c4[1] += arrived;
    c4[2] += cands;
    c4[3] += entered;
}

// Transfers of step t for link / origin node i (every thread of the block calls).
__device__ __forceinline__ void step_b(const DevSim &d, int i, int t) {
    int c4[4] = {0, 0, 0, 0};
    step_b_core(d, i, t, c4);
    __shared__ int smem[8];
    block_count(c4[0], &d.step_delta[4 * t + 0], smem);
    block_count(c4[1], &d.step_delta[4 * t + 1], smem);
    block_count(c4[2], &d.step_delta[4 * t + 2], smem);
    block_count(c4[3], &d.step_delta[4 * t + 3], smem);
}


__global__ void __launch_bounds__(256) k_step_b(DevSim d, int t) {
    step_b(d, blockIdx.x * blockDim.x + threadIdx.x, t);
}

// ---------------------------------------------------------------------------
// Batched launches: one kernel per phase over the blocks of many simulator
// instances (members), each block belonging to one member.  Members carry their
// own step counter and mode in device memory, so that they can have different
// horizons and join or leave at step boundaries.
// ---------------------------------------------------------------------------
constexpr int kModeRun = 0, kModeFinal = 1, kModeDone = 2;

__device__ __forceinline__ void load_member(DevSim &sd, const DevSim *ds, int m) {
    const int nw = (int)(sizeof(DevSim) / sizeof(int));
    for (int k = threadIdx.x; k < nw; k += blockDim.x) reinterpret_cast<int *>(&sd)[k] = reinterpret_cast<const int *>(ds + m)[k];
    __syncthreads();
}

__global__ void __launch_bounds__(kBlockA, 6) k_batch_a(const DevSim *ds, const int2 *bmap, const int *tvec,
                                                        const int *mode) {
    extern __shared__ float xs[];
    __shared__ DevSim sd;
    const int2 m = bmap[blockIdx.x];
    const int md = mode[m.x];
    if (md == kModeDone) return;
    load_member(sd, ds, m.x);
    step_block<false>(sd, m.y, tvec[m.x], md == kModeFinal, xs);
}

__global__ void __launch_bounds__(256) k_batch_b(const DevSim *ds, const int2 *bmap, const int *tvec, const int *mode) {
    __shared__ DevSim sd;
    const int2 m = bmap[blockIdx.x];
    if (mode[m.x] != kModeRun) return;
    load_member(sd, ds, m.x);
    step_b(sd, m.y * 256 + (int)threadIdx.x, tvec[m.x]);
}

// after each batched step: running members advance; a member reaching its
// horizon closes its last bin in the next step's pass, then stops
__global__ void k_batch_tick(int n, int *tvec, const int *Tvec, int *mode) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int md = mode[m];
    if (md == kModeRun) {
        const int t = tvec[m] + 1;
        tvec[m] = t;
        if (t >= Tvec[m]) mode[m] = kModeFinal;
    } else if (md == kModeFinal) {
        mode[m] = kModeDone;
    }
}

// checkpoint of the members recording a tape (every K steps, before the step)
struct CkDev {
    int K, L, S, V, N;
    int4 *lq, *lstat;
    int *vac, *sentry, *fifo, *vstate;
    float *pos;
    int2 *saux;
    longlong2 *lpos;
};

// checkpoint t / K of one member, by threads i0, i0 + stride, ...
__device__ __forceinline__ void ckpt_member(const DevSim &d, const CkDev &c, int t, size_t i0, size_t stride) {
    const size_t s = t / c.K;
    const float *pc = (t & 1) ? d.pos1 : d.pos0;
    for (size_t i = i0; i < (size_t)c.S; i += stride) {
        c.pos[s * c.S + i] = pc[i];
        c.saux[s * c.S + i] = d.saux[i];
        c.sentry[s * c.S + i] = d.sentry[i];
    }
    for (size_t i = i0; i < (size_t)c.L; i += stride) {
        c.lq[s * c.L + i] = d.lq[i];
        c.lstat[s * c.L + i] = d.lstat[i];
        c.vac[s * c.L + i] = d.vac[i];
        c.lpos[s * c.L + i] = d.lpos[i];
    }
    for (size_t i = i0; i < (size_t)c.V; i += stride) c.fifo[s * c.V + i] = d.fifo_ptr[i];
    for (size_t i = i0; i < (size_t)c.N; i += stride) c.vstate[s * c.N + i] = d.vstate[i];
}

// the dynamic state from checkpoint t / K (the inverse of ckpt_member)
__device__ __forceinline__ void restore_member(const DevSim &d, const CkDev &c, int t, size_t i0, size_t stride) {
    const size_t s = t / c.K;
    float *pc = (t & 1) ? d.pos1 : d.pos0;
    for (size_t i = i0; i < (size_t)c.S; i += stride) {
        pc[i] = c.pos[s * c.S + i];
        d.saux[i] = c.saux[s * c.S + i];
        d.sentry[i] = c.sentry[s * c.S + i];
    }
    for (size_t i = i0; i < (size_t)c.L; i += stride) {
        d.lq[i] = c.lq[s * c.L + i];
        d.lstat[i] = c.lstat[s * c.L + i];
        d.vac[i] = c.vac[s * c.L + i];
        d.lpos[i] = c.lpos[s * c.L + i];
    }
    for (size_t i = i0; i < (size_t)c.V; i += stride) d.fifo_ptr[i] = c.fifo[s * c.V + i];
    for (size_t i = i0; i < (size_t)c.N; i += stride) d.vstate[i] = c.vstate[s * c.N + i];
}

// one instance: save (or restore) checkpoint t / K in one launch
__global__ void k_ckpt(DevSim d, CkDev c, int t, int save) {
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if (save) ckpt_member(d, c, t, i0, stride);
    else restore_member(d, c, t, i0, stride);
}

__global__ void k_batch_ckpt(const DevSim *ds, const CkDev *cks, const int *tvec, const int *mode) {
    const int m = blockIdx.y;
    const CkDev c = cks[m];
    if (c.K <= 0 || mode[m] != kModeRun) return;
    const int t = tvec[m];
    if (t % c.K != 0) return;
    ckpt_member(ds[m], c, t, blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

}  // namespace ts
