// Batched persistent executor (sm_103a): many simulator instances (members)
// advanced by one cooperative launch for any number of steps.
//
// The two-kernel batch (k_batch_a / k_batch_b) runs the node model in blocks of
// at most 64 links with four block barriers per step.  A batch of tens of
// scenarios on a city network has millions of links, most of them empty or
// nearly so, and there it is bound by the latency of dozens of waves of such
// blocks.  Here one warp takes 32 links (lane = link) through the whole node
// model with warp-synchronous code only, so that each SM keeps 1,024 links in
// flight and no block barrier holds the warps of a CTA.  Per step:
//   phase K  (only at steps where a member checkpoints) the checkpoints;
//   phase A  link items: queue state, outflow credit, candidate, its choice slots
//            and keys, Newell car-following of the item's vehicles (lanes over
//            queue positions, headways by shuffle), observation sums, argmax,
//            merge atomicMax, next-step bits and records -- the arithmetic of
//            step_block, element for element; origin-node items: the head of
//            each origin queue (a virtual inflow link of length 0);
//   phase B  the transfers of every link and origin node (step_b_core);
// each phase closed by a bounded grid barrier.  Members keep their own step and
// mode: the phase a member is in at step s of the launch follows from its step,
// mode and horizon at the start of the launch.
#pragma once
#include "ts_persist.cuh"

namespace ts {

constexpr int kBT = 1024;                 // threads per CTA (one CTA per SM)
constexpr int kBW = kBT / 32;             // warps per CTA
constexpr int kBMaxMembers = 1024;        // members of one launch (shared-memory table)
constexpr int kItemNode = 1 << 30;        // item flag: origin nodes instead of links

struct BArgs {
    const DevSim *ds;
    const CkDev *ck;
    const int2 *itA;                      // [nA] (member, first link) or (member, first node | kItemNode)
    const int2 *itB;                      // [nB] (member, first element of [0, L + V))
    const unsigned char *ckstep;          // [n_steps] 1 where some member checkpoints
    int nA, nB;
    int *tvec, *Tvec, *mode;
    int n, n_steps;
    unsigned *bar;                        // grid-barrier counter, zero at launch
    int *berr;                            // SIM_ETIMEOUT once a barrier gave up
    int bar_extra;                        // test hook: arrivals every barrier waits for in vain
};

struct BWarpSmem {                        // one per warp; rows indexed by lane (= link)
    float4 lo[32][kMaxSlotsStaged];       // choice slots of the candidate
    float key[32][kMaxSlotsStaged];
    int vacm[32][kMaxSlotsStaged];
    float4 x4[32];                        // new positions of vehicles 0, 1, n-2, n-1
    int4 stat[32];
    longlong2 ps[32];
    unsigned long long psum[32];          // position sum (observation)
    int past[32];                         // vehicles past the midpoint (observation)
};

inline size_t b_dyn_bytes(int n_members) {
    return (size_t)kBW * sizeof(BWarpSmem) + (size_t)n_members * sizeof(int4);
}

// Phase of a member at step s of the launch from (t0, mode0, T) at its start;
// t = the member's step.  Matches the two-kernel batch: run steps t0 .. T-1,
// then one observation-only pass at t = T that closes the last bin.
__device__ __forceinline__ int bphase(int4 mb, int s, int &t) {
    const int t0 = mb.x, mode0 = mb.y, T = mb.z;
    t = t0;
    if (mode0 == kModeDone) return kModeDone;
    if (mode0 == kModeFinal) return s == 0 ? kModeFinal : kModeDone;
    const int r = T - t0;
    if (s < r) { t = t0 + s; return kModeRun; }
    t = T;
    return s == r ? kModeFinal : kModeDone;
}

// Bounded grid barrier (same protocol as the single-instance executor).
__device__ __forceinline__ bool bsync(const BArgs &a, unsigned target, int *stop) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(a.bar) : "memory");
        const unsigned long long t_start = global_ns();
        int ok = 1;
        for (unsigned it = 0;; ++it) {
            if (ld_acquire_gpu(a.bar) >= target) break;
            if ((it & 255u) == 255u) {
                if (it >= (1u << 22) || global_ns() - t_start > 2000000000ull || __ldcg(a.berr) != 0) {
                    atomicCAS(a.berr, 0, SIM_ETIMEOUT);
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

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Element e of the concatenated queues of a link item: the lane of its link
// (the last lane whose offset is <= e), its queue position and slot.
struct BElem {
    int li, k, lqy, slot;
    float gx, gy, gz, gw;
    bool act;
};
__device__ __forceinline__ BElem b_elem(int e, int total, int excl, int4 q, int4 st, float4 g) {
    BElem r;
    r.act = e < total;
    int li = 0;
#pragma unroll
    for (int stp = 16; stp >= 1; stp >>= 1)
        if (__shfl_sync(kFull, excl, li + stp) <= e) li += stp;
    r.li = li;
    r.k = e - __shfl_sync(kFull, excl, li);
    const int lqx = __shfl_sync(kFull, q.x, li);
    r.lqy = __shfl_sync(kFull, q.y, li);
    const int lbase = __shfl_sync(kFull, st.x, li);
    const int lcap = __shfl_sync(kFull, st.y, li);
    r.gx = __shfl_sync(kFull, g.x, li);
    r.gy = __shfl_sync(kFull, g.y, li);
    r.gz = __shfl_sync(kFull, g.z, li);
    r.gw = __shfl_sync(kFull, g.w, li);
    int idx = lqx + r.k;
    if (idx >= lcap) idx -= lcap;
    r.slot = lbase + idx;
    return r;
}

// Phase A, links [j0, j0 + 32) of member d; lane = link.  obs_only: the pass
// that closes the last bin (observation outputs only).  A warp issues in
// order and waits at the first use of a loaded value, so the loads go in three
// rounds, each issued whole before anything waits on it: link data; leader,
// choice slots, statistics (copied asynchronously into shared memory) and the
// first 32 positions; destination features and the targets' flags, while the
// Gumbel noise is drawn.
__device__ __forceinline__ void bwarp_links(const DevSim &d, int j0, int t, bool obs_only, BWarpSmem &S) {
    const int lane = threadIdx.x & 31;
    const int nl = min(32, d.L - j0);
    const bool valid = lane < nl;
    const int j = j0 + lane;
    const int p = t & 1;
    const float *pc = p ? d.pos1 : d.pos0;
    float *pn = p ? d.pos0 : d.pos1;
    const bool obs = obs_only || (t > 0 && t % d.obs_every == 0);
    __syncwarp();
    // load round 1: queue state and link data
    int4 q = make_int4(0, 0, 0, 0), st = make_int4(0, 0, 0, 0), nd = make_int4(0, 0, 0, 0);
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int flags = 0, eb = 0;
    float alpha = 0.0f;
    if (valid) {
        q = d.lq[j];
        st = d.lst[j];
        flags = d.vac[j];
        g = d.geo[j];
        nd = d.lnode[j];
        alpha = d.alpha[j];
        eb = d.ebits[j];
    }
    const int credit = min(q.z + st.z, st.w);
    const bool cand = valid && !obs_only && q.y > 0 && (flags & kFlagArrive) && credit >= d.dn_fx;
    const int deg = nd.w - nd.z;
    const int n = valid ? q.y : 0;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const int excl = incl - n;
    const int total = __shfl_sync(kFull, incl, 31);
    // load round 2: leader and choice slots of a candidate, bin statistics, the
    // positions of the first 32 vehicles of the item
    int2 lead = make_int2(-1, -1);
    int ent = 0;
    if (cand) {
        lead = d.saux[st.x + q.x];
        ent = d.sentry[st.x + q.x];
#pragma unroll
        for (int k = 0; k < kMaxSlotsStaged; ++k)
            if (k < deg) cp_async16(&S.lo[lane][k], d.loinfo + nd.z + k);
    }
    if (valid && (n > 0 || obs)) {
        cp_async16(&S.stat[lane], d.lstat + j);
        cp_async16(&S.ps[lane], d.lpos + j);
    }
    BElem E = b_elem(lane, total, excl, q, st, g);
    float x = E.act ? pc[E.slot] : 0.0f;
    S.past[lane] = 0;
    S.psum[lane] = 0ull;
    cp_async_wait_all();
    // load round 3: utility + Gumbel keys of the candidate's slots
    float mkey = 0.0f;
    if (cand) {
        const bool choose_here = nd.y != lead.y;
        float df[kMaxSlotsStaged];
        int vm[kMaxSlotsStaged];
#pragma unroll
        for (int k = 0; k < kMaxSlotsStaged; ++k) {
            df[k] = 0.0f;
            vm[k] = 0;
            if (choose_here && k < deg) {
                const float4 e = S.lo[lane][k];
                df[k] = d.dest_feat[(size_t)lead.y * d.V + __float_as_int(e.z)];
                vm[k] = d.vac[__float_as_int(e.w)];
            }
        }
        mkey = __fadd_rn(alpha, gumbel(d.key0, d.key1, lead.x, t, 1, 0));
        if (choose_here) {               // slots 0..3 are the four words of one Philox block
            const uint4 o = gumbel_block(d.key0, d.key1, lead.x, t, 0, 0);
#pragma unroll
            for (int k = 0; k < kMaxSlotsStaged; ++k) {
                if (k < deg) {
                    const float gk = gumbel_of_word(k == 0 ? o.x : k == 1 ? o.y : k == 2 ? o.z : o.w);
                    const float4 e = S.lo[lane][k];
                    S.key[lane][k] = __fadd_rn(__fadd_rn(e.x, __fmul_rn(e.y, df[k])), gk);
                    S.vacm[lane][k] = vm[k] & kFlagVacant;
                }
            }
        }
    }
    // car-following over the item's vehicles (chunks of 32 of the concatenated
    // queues; the vehicle ahead by shuffle, across chunks by carry)
    float carry = 0.0f;
    for (int base = 0; base < total; base += 32) {
        if (base > 0) {
            E = b_elem(base + lane, total, excl, q, st, g);
            x = E.act ? pc[E.slot] : 0.0f;
        }
        const int li = E.li, k = E.k;
        float xp = __shfl_up_sync(kFull, x, 1);
        if (lane == 0) xp = carry;
        carry = __shfl_sync(kFull, x, 31);
        if (E.act && !obs_only) {
            const float h = (k == 0) ? d.M : __fsub_rn(xp, x);
            int tag;
            const float xn = newell(x, h, E.gx, E.gy, E.gz, E.gw, tag);
            pn[E.slot] = xn;
            if (k == 0) S.x4[li].x = xn;
            if (k == 1) S.x4[li].y = xn;
            if (k == E.lqy - 2) S.x4[li].z = xn;
            if (k == E.lqy - 1) S.x4[li].w = xn;
        }
        if (obs) {                       // warp-uniform: midpoint count and position sum per link
            const unsigned seg = __match_any_sync(kFull, E.act ? li : -1);
            const unsigned past = E.act && x >= __fmul_rn(E.gx, 0.5f) ? 1u : 0u;
            const unsigned sp = __reduce_add_sync(seg, past);
            const long long xf = E.act ? pos_fx(x) : 0;
            const unsigned slo = __reduce_add_sync(seg, (unsigned)(xf & 0xffffffll));
            const unsigned shi = __reduce_add_sync(seg, (unsigned)(xf >> 24));
            if (E.act && lane == __ffs(seg) - 1) {
                S.past[li] += (int)sp;
                S.psum[li] += (unsigned long long)slo + ((unsigned long long)shi << 24);
            }
        }
    }
    __syncwarp();
    // observation, choice, merge, next-step flags, record
    if (!valid) return;
    if (n == 0 && !obs) {                // empty link: credit, and the static bits of an empty queue
        d.lq[j].z = credit;
        d.crec[j] = make_int4(-1, kTgtNone, eb, 0);
        return;
    }
    int4 stat = S.stat[lane];
    longlong2 ps = S.ps[lane];
    if (obs) {
        const int bin = (t - 1) / d.obs_every;
        const size_t o = (size_t)bin * d.L + j;
        const int C = q.w + S.past[lane];
        d.out_counts[o] = C - stat.w;
        const long long pnow = (long long)S.psum[lane];
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
    int tgt = kTgtNone;
    if (cand) {
        if (nd.y == lead.y) {
            tgt = kTgtSink;
        } else {
            tgt = choose(d, S.lo[lane], S.key[lane], S.vacm[lane], d.loinfo + nd.z, deg, lead.y, lead.x, t);
            if (tgt >= 0) atomicMax(p ? &d.W1[tgt] : &d.W0[tgt], merge_word(mkey, lead.x));
        }
    }
    d.lq[j].z = credit;
    const float M = d.M;
    const float4 x4 = S.x4[lane];
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
    d.crec[j] = make_int4(cand ? lead.x : -1, cand ? tgt : kTgtNone, (ent << 8) | bits, __float_as_int(x0));
}

// Phase A, origin queues of nodes [n0, n0 + 32) of member d; lane = node.
__device__ __forceinline__ void bwarp_nodes(const DevSim &d, int n0, int t, BWarpSmem &S) {
    const int lane = threadIdx.x & 31;
    const int n = n0 + lane;
    __syncwarp();
    if (n >= d.V) return;
    const int p = t & 1;
    const int4 nq = make_int4(d.fifo_ptr[n], d.fifo_end[n], d.no_ptr[n], d.no_ptr[n + 1]);
    const int zone = d.node_zone[n];
    const int deg = nq.w - nq.z;
    int2 lead = make_int2(-1, -1);
    if (nq.x < nq.y) {                   // loads issued before the departure test
        const int dep = d.fifo_dep[nq.x];
        const int2 head = d.fifo_list[nq.x];
#pragma unroll
        for (int k = 0; k < kMaxSlotsStaged; ++k)
            if (k < deg) S.lo[lane][k] = d.noinfo[nq.z + k];
        if (dep <= t) lead = head;
    }
    int tgt = kTgtNone;
    if (lead.x >= 0) {
        if (zone == lead.y) {
            tgt = kTgtSink;
        } else {
            const float mkey = __fadd_rn(d.alpha[d.L], gumbel(d.key0, d.key1, lead.x, t, 1, 0));
#pragma unroll
            for (int k = 0; k < kMaxSlotsStaged; ++k) {
                if (k < deg) {
                    const float4 e = S.lo[lane][k];
                    S.key[lane][k] = choice_key(d, e, lead.y, lead.x, t, k);
                    S.vacm[lane][k] = d.vac[__float_as_int(e.w)] & kFlagVacant;
                }
            }
            tgt = choose(d, S.lo[lane], S.key[lane], S.vacm[lane], d.noinfo + nq.z, deg, lead.y, lead.x, t);
            if (tgt >= 0) atomicMax(p ? &d.W1[tgt] : &d.W0[tgt], merge_word(mkey, lead.x));
        }
    }
    d.nrec[n] = make_int2(lead.x, tgt);
}

__global__ void __launch_bounds__(kBT, 1) k_batch_persist(BArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    BWarpSmem *WS = reinterpret_cast<BWarpSmem *>(bsm);
    int4 *mem = reinterpret_cast<int4 *>(bsm + (size_t)kBW * sizeof(BWarpSmem));
    __shared__ int stop;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int m = tid; m < a.n; m += kBT) mem[m] = make_int4(a.tvec[m], a.mode[m], a.Tvec[m], a.ck[m].K);
    __syncthreads();
    BWarpSmem &S = WS[tid >> 5];
    const int gw = blockIdx.x * kBW + (tid >> 5), nw = gridDim.x * kBW;
    const size_t gtid = (size_t)blockIdx.x * kBT + tid, gstride = (size_t)gridDim.x * kBT;
    unsigned epoch = 0;
    for (int s = 0; s < a.n_steps; ++s) {
        if (a.ckstep[s]) {               // checkpoints of the step (before it)
            for (int m = 0; m < a.n; ++m) {
                int t;
                const int4 mb = mem[m];
                if (mb.w > 0 && bphase(mb, s, t) == kModeRun && t % mb.w == 0) ckpt_member(a.ds[m], a.ck[m], t, gtid, gstride);
            }
            if (!bsync(a, ++epoch * gridDim.x + (unsigned)a.bar_extra, &stop)) return;
        }
        for (int it = gw; it < a.nA; it += nw) {
            const int2 w = a.itA[it];
            int t;
            const int ph = bphase(mem[w.x], s, t);
            if (ph == kModeDone) continue;
            const DevSim &d = a.ds[w.x];
            if (w.y & kItemNode) {
                if (ph == kModeRun) bwarp_nodes(d, w.y & ~kItemNode, t, S);
            } else {
                bwarp_links(d, w.y, t, ph == kModeFinal, S);
            }
        }
        if (!bsync(a, ++epoch * gridDim.x + (unsigned)a.bar_extra, &stop)) return;
        for (int it = gw; it < a.nB; it += nw) {
            const int2 w = a.itB[it];
            int t;
            if (bphase(mem[w.x], s, t) != kModeRun) continue;
            const DevSim &d = a.ds[w.x];
            int c4[4] = {0, 0, 0, 0};
            step_b_core(d, w.y + lane, t, c4);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int v = warp_sum(c4[c]);
                if (lane == 0 && v) atomicAdd(&d.step_delta[4 * t + c], v);
            }
        }
        if (!bsync(a, ++epoch * gridDim.x + (unsigned)a.bar_extra, &stop)) return;
    }
    if (blockIdx.x == 0) {               // members' step and mode after the launch
        for (int m = tid; m < a.n; m += kBT) {
            int t;
            const int ph = bphase(mem[m], a.n_steps, t);
            a.tvec[m] = t;
            a.mode[m] = ph;
        }
    }
}

}  // namespace ts
