// Persistent forward executor (sm_103a): a run of steps in ONE cooperative
// launch, one CTA of kPT threads per SM, each CTA owning a fixed group of
// consecutive links and a fixed range of origin queues for the whole launch.
//
// The queues of a CTA's links stay in its shared memory for the whole launch
// (FIFO rings, leader first, one float position per slot: the order of SI-A's
// argsort, maintained instead of re-sorted because vehicles never overtake), so
// that the car-following update reads and writes no global memory.  Across
// CTAs, the node model of SI-B couples links only through
//   * the merge words W[target] (64-bit atomicMax of alpha + g', ~vehicle),
//     three buffers indexed by step mod 3, and
//   * each link's record of the step (candidate, target, next-step vacancy /
//     arrival bits for the four (pop, push) outcomes), two buffers by parity,
// from which any CTA derives the vacancy of any link for the next step without
// waiting for the link's owner to apply its transfers.  One grid-wide barrier
// per step therefore suffices: epoch t = [transfers of step t-1 for own links]
// [step t: credit, candidates, car-following, link choice, merge] barrier.
//
// Every floating-point operation is the one of the two-kernel path (same device
// functions, same order), so both executors give bit-identical results.
// Every wait is bounded: a barrier that does not complete within ~2 s records
// SIM_ETIMEOUT and every CTA returns.
#pragma once
#include "ts_step.cuh"

namespace ts {

constexpr int kPT = 1024;        // threads per CTA
constexpr int kPLinks = 320;     // links per CTA at most
constexpr int kPNodes = 256;     // origin queues per CTA at most
constexpr int kPU = 4;           // car-following elements per thread per chunk
constexpr int kPSlot = 4;        // choice slots per candidate evaluated in parallel

struct PArgs {
    const int *grp_links;          // [G + 1] first link of each CTA's group
    int npg;                       // origin queues per CTA
    unsigned long long *W3;        // [3 L] merge words by step mod 3
    int4 *crec2;                   // [2 L] link records by step parity
    unsigned *bar;                 // grid barrier counter (zero at launch)
    int t0, t1;                    // steps [t0, t1)
    int final_obs;                 // close the last bin at t1 (observation-only pass)
};

struct PSmem {
    int4 q[kPLinks];               // queue head, length, credit, exits
    int4 st[kPLinks];              // global slot base, capacity, q_fx, credit cap
    float4 g[kPLinks];             // length, u dt, s, tag band
    int4 nd[kPLinks];              // head node, head zone, choice begin/end
    int4 stat[kPLinks];            // open-bin statistics
    int4 cr[kPLinks];              // record of the step (candidate, target, entry << 8 | bits, x0)
    float4 x4[kPLinks];            // new positions of vehicles 0, 1, n-2, n-1
    int2 lead[kPLinks];            // candidate (vehicle, zone)
    int flags[kPLinks];            // vacancy / arrival for the coming step
    int off[kPLinks + 1];          // first element of each link in the block's element order
    int past[kPLinks];             // vehicles past the midpoint (observation)
    float mkey[kPLinks];           // merge key alpha + g' of the candidate
    unsigned long long psum[kPLinks];
    float key[kPLinks][kPSlot];    // utility + Gumbel of each choice slot
    int tv[kPLinks][kPSlot];       // target << 1 | vacant
    int4 nq[kPNodes];              // next vehicle, end of queue, out-links begin/end
    int2 nlead[kPNodes];
    int2 nrec[kPNodes];            // (candidate, target) of the step
    int nzone[kPNodes];
    float nmkey[kPNodes];
    float nkey[kPNodes][kPSlot];
    int ntv[kPNodes][kPSlot];
    int wsum[32], wpre[32];
    int cnt[4];                    // step counters: releases, arrivals, candidates, entries
    float carry[2];                // old position of the last element of a chunk, by chunk parity
    int total;
    int stop;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number `target / gridDim.x` (counter never reset inside a
// launch).  Bounded: gives up after ~2 s or 2^22 polls, or as soon as another
// CTA has recorded a timeout; returns false then (every thread of the CTA).
__device__ __forceinline__ bool grid_sync(const DevSim &d, unsigned *bar, unsigned target, int t, int *stop) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
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
            __nanosleep(20);
        }
        __threadfence();
        *stop = !ok;
    }
    __syncthreads();
    return *stop == 0;
}

// Vacancy / arrival flags of link m for step t, from its record of step t-1
// and the merge words of step t-1 (what its owner will apply).
__device__ __forceinline__ int derived_flags(const int4 *Cp, const unsigned long long *Wp, int m) {
    const int4 c = __ldcg(Cp + m);
    bool pop = c.y == kTgtSink;
    if (c.y >= 0) {
        const unsigned long long w = __ldcg(Wp + c.y);
        pop = w != 0ull && merge_vid(w) == c.x;
    }
    const bool push = __ldcg(Wp + m) != 0ull;
    const int o = (pop ? 1 : 0) | (push ? 2 : 0);
    return ((c.z >> o) & 1) | (((c.z >> (4 + o)) & 1) << 1);
}

__device__ __forceinline__ int vacant_of(const DevSim &d, bool first, const int4 *Cp, const unsigned long long *Wp,
                                         int m) {
    return (first ? __ldcg(d.vac + m) : derived_flags(Cp, Wp, m)) & kFlagVacant;
}

// argmax of the staged keys (ties to the lowest slot); slots past the stage
// are evaluated inline.  Returns the target or kTgtBlocked.
__device__ __forceinline__ int p_choose(const DevSim &d, bool first, const int4 *Cp, const unsigned long long *Wp,
                                        const float *key, const int *tv, const float4 *info, int deg, int zone,
                                        int vid, int t) {
    float bk = -INFINITY;
    int bm = -1, bv = 0;
    for (int k = 0; k < deg; ++k) {
        float kk;
        int m, vm;
        if (k < kPSlot) {
            kk = key[k];
            m = tv[k] >> 1;
            vm = tv[k] & 1;
        } else {
            const float4 e = info[k];
            kk = choice_key(d, e, zone, vid, t, k);
            m = __float_as_int(e.w);
            vm = vacant_of(d, first, Cp, Wp, m);
        }
        if (bm < 0 || kk > bk) { bk = kk; bm = m; bv = vm; }
    }
    return bv ? bm : kTgtBlocked;
}

// Transfers of step tb for the CTA's links and origin queues (SI-B Eq.
// transfer): pop the leader that won its merge or left to its destination, push
// the merge winner at x = 0, then the flags of step tb + 1.
__device__ __forceinline__ void p_transfers(const DevSim &d, const PArgs &a, PSmem &S, float *P, int j0, int nl,
                                            int nn, int base0, int tb) {
    const unsigned long long *Wb = a.W3 + (size_t)(tb % 3) * d.L;
    unsigned long long *Wc = a.W3 + (size_t)((tb + 2) % 3) * d.L;    // words of step tb + 2
    int released = 0, arrived = 0, cands = 0, entered = 0;
    for (int li = threadIdx.x; li < nl; li += kPT) {
        const int j = j0 + li;
        int4 q = S.q[li];
        const int4 st = S.st[li];
        const int4 c = S.cr[li];
        const unsigned long long win = __ldcg(Wb + j);
        bool pop = false;
        cands += c.x >= 0;
        if (c.y == kTgtSink) {
            pop = true;
            d.vstate[c.x] = kVehArrived;
            arrived += 1;
        } else if (c.y >= 0) {
            const unsigned long long w = __ldcg(Wb + c.y);
            pop = w != 0ull && merge_vid(w) == c.x;
        }
        if (pop) {
            int4 stat = S.stat[li];
            stat.y += tb + 1 - (c.z >> 8);
            stat.z += 1;
            S.stat[li] = stat;
            longlong2 ps = d.lpos[j];
            ps.y += pos_fx(__int_as_float(c.w));
            d.lpos[j] = ps;
            q.x = (q.x + 1 == st.y) ? 0 : q.x + 1;
            q.y -= 1;
            q.z -= d.dn_fx;
            q.w += 1;
        }
        const bool push = win != 0ull;
        if (push) {
            const int v = merge_vid(win);
            if (q.y >= st.y) {
                set_error(d, SIM_EOVERFLOW, j, tb);
            } else {
                int idx = q.x + q.y;
                if (idx >= st.y) idx -= st.y;
                P[st.x - base0 + idx] = 0.0f;
                d.saux[st.x + idx] = make_int2(v, d.dest_zone[v]);
                d.sentry[st.x + idx] = tb + 1;
                q.y += 1;
                d.vstate[v] = j;
                entered += 1;
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
        S.q[li] = q;
        const int o = (pop ? 1 : 0) | (push ? 2 : 0);
        S.flags[li] = ((c.z >> o) & 1) | (((c.z >> (4 + o)) & 1) << 1);
        Wc[j] = 0ull;
    }
    for (int ni = threadIdx.x; ni < nn; ni += kPT) {
        const int2 c = S.nrec[ni];
        cands += c.x >= 0;
        if (c.y == kTgtSink) {
            S.nq[ni].x += 1;
            d.vstate[c.x] = kVehArrived;
            released += 1;
            arrived += 1;
        } else if (c.y >= 0) {
            const unsigned long long w = __ldcg(Wb + c.y);
            if (w != 0ull && merge_vid(w) == c.x) { S.nq[ni].x += 1; released += 1; }
        }
    }
    released = warp_sum(released);
    arrived = warp_sum(arrived);
    cands = warp_sum(cands);
    entered = warp_sum(entered);
    if ((threadIdx.x & 31) == 0) {
        if (released) atomicAdd(&S.cnt[0], released);
        if (arrived) atomicAdd(&S.cnt[1], arrived);
        if (cands) atomicAdd(&S.cnt[2], cands);
        if (entered) atomicAdd(&S.cnt[3], entered);
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int v = S.cnt[threadIdx.x];
        if (v) atomicAdd(&d.step_delta[4 * tb + threadIdx.x], v);
        S.cnt[threadIdx.x] = 0;
    }
}

// Step t for the CTA's links and origin queues: credit and candidates, Newell
// car-following in shared memory, observation at bin ends, link choice and
// merge.  obs_only: only close the bin ending at t.
__device__ __forceinline__ void p_step(const DevSim &d, const PArgs &a, PSmem &S, float *P, int j0, int nl, int n0,
                                       int nn, int base0, int t, bool first, bool obs_only) {
    const int tid = threadIdx.x, lane = tid & 31;
    const bool obs = obs_only || (t > 0 && t % d.obs_every == 0);
    if (obs_only) nn = 0;
    // ---------------- credit, candidates, queue-length scan ----------------
    for (int li = tid; li < nl; li += kPT) {
        S.past[li] = 0;
        S.psum[li] = 0ull;
        if (obs_only) continue;             // the records of the last step stay
        const int4 q = S.q[li];
        const int4 st = S.st[li];
        const int credit = min(q.z + st.z, st.w);
        S.q[li].z = credit;
        const bool cand = (S.flags[li] & kFlagArrive) && credit >= d.dn_fx;
        int2 lead = make_int2(-1, -1);
        int ent = 0;
        if (cand) {
            lead = d.saux[st.x + q.x];
            ent = d.sentry[st.x + q.x];
        }
        S.lead[li] = lead;
        S.cr[li] = make_int4(cand ? lead.x : -1, kTgtNone, ent, 0);
    }
    for (int ni = tid; ni < nn; ni += kPT) {
        const int4 nq = S.nq[ni];
        int2 lead = make_int2(-1, -1);
        if (nq.x < nq.y) {
            const int dep = d.fifo_dep[nq.x];
            const int2 head = d.fifo_list[nq.x];
            if (dep <= t) lead = head;
        }
        S.nlead[ni] = lead;
    }
    if (tid < kPLinks) {                    // exclusive scan of queue lengths, per warp
        const int v = tid < nl ? S.q[tid].y : 0;
        int s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane == 31) S.wsum[tid >> 5] = s;
        S.off[tid] = s - v;
    }
    __syncthreads();
    if (tid < 32) {
        const int v = tid < kPLinks / 32 ? S.wsum[tid] : 0;
        int s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        S.wpre[tid] = s - v;
        if (tid == 31) S.total = s;
    }
    __syncthreads();
    if (tid < nl) S.off[tid] += S.wpre[tid >> 5];
    if (tid == 0) S.off[nl] = S.total;
    __syncthreads();
    const int total = S.total;
    const int4 *Cp = a.crec2 + (size_t)((t + 1) & 1) * d.L;                 // records of step t-1
    const unsigned long long *Wp = a.W3 + (size_t)((t + 2) % 3) * d.L;     // words of step t-1
    // ---------------- link-choice and merge keys of the candidates ----------------
    if (!obs_only) {
        for (int c = tid; c < (nl + nn) * kPSlot; c += kPT) {
            const int r = c / kPSlot, k = c % kPSlot;
            if (r < nl) {
                const int2 lead = S.lead[r];
                if (lead.x < 0 || S.cr[r].x < 0) continue;
                const int4 nd = S.nd[r];
                if (k == 0) S.mkey[r] = __fadd_rn(d.alpha[j0 + r], gumbel(d.key0, d.key1, lead.x, t, 1, 0));
                if (k >= nd.w - nd.z || nd.y == lead.y) continue;
                const float4 e = d.loinfo[nd.z + k];
                const int m = __float_as_int(e.w);
                S.key[r][k] = choice_key(d, e, lead.y, lead.x, t, k);
                S.tv[r][k] = (m << 1) | vacant_of(d, first, Cp, Wp, m);
            } else {
                const int q = r - nl;
                const int2 lead = S.nlead[q];
                if (lead.x < 0) continue;
                const int4 nq = S.nq[q];
                if (k == 0) S.nmkey[q] = __fadd_rn(d.alpha[d.L], gumbel(d.key0, d.key1, lead.x, t, 1, 0));
                if (k >= nq.w - nq.z || S.nzone[q] == lead.y) continue;
                const float4 e = d.noinfo[nq.z + k];
                const int m = __float_as_int(e.w);
                S.nkey[q][k] = choice_key(d, e, lead.y, lead.x, t, k);
                S.ntv[q][k] = (m << 1) | vacant_of(d, first, Cp, Wp, m);
            }
        }
    }
    // ---------------- car-following in shared memory, chunk by chunk ----------------
    // Warp w of a chunk handles elements [cb + 32 kPU w, cb + 32 kPU (w + 1)),
    // lane-interleaved; new positions are written after every thread of the
    // chunk has read its time-t headway.
    const float M = d.M;
    for (int cb = 0, ci = 0; cb < total; cb += kPT * kPU, ++ci) {
        const int wbase = cb + (tid >> 5) * 32 * kPU;
        float xn[kPU];
        int sidx[kPU];
        int li = link_of(S.off, nl, min(wbase + lane, total - 1));
#pragma unroll
        for (int u = 0; u < kPU; ++u) {
            const int e = wbase + u * 32 + lane;
            const bool act = e < total;
            float x = 0.0f;
            sidx[u] = -1;
            xn[u] = 0.0f;
            if (act) {
                while (S.off[li + 1] <= e) ++li;
                const int k = e - S.off[li];
                const int4 q = S.q[li], st = S.st[li];
                const int lb = st.x - base0;
                int idx = q.x + k;
                if (idx >= st.y) idx -= st.y;
                x = P[lb + idx];
                if (e == cb + kPT * kPU - 1) S.carry[(ci + 1) & 1] = x;
                if (!obs_only) {
                    float h;
                    if (k == 0) {
                        h = M;
                    } else if (e == cb) {
                        h = __fsub_rn(S.carry[ci & 1], x);
                    } else {
                        const int ip = idx == 0 ? st.y - 1 : idx - 1;
                        h = __fsub_rn(P[lb + ip], x);
                    }
                    const float4 g = S.g[li];
                    int tag;
                    xn[u] = newell(x, h, g.x, g.y, g.z, g.w, tag);
                    sidx[u] = lb + idx;
                    if (k == 0) S.x4[li].x = xn[u];
                    if (k == 1) S.x4[li].y = xn[u];
                    if (k == q.y - 2) S.x4[li].z = xn[u];
                    if (k == q.y - 1) S.x4[li].w = xn[u];
                }
            }
            if (obs) {      // block-uniform: midpoint count and position sum per link
                const unsigned seg = __match_any_sync(kFull, act ? li : -1);
                const unsigned past = act && x >= __fmul_rn(S.g[li].x, 0.5f) ? 1u : 0u;
                const unsigned sp = __reduce_add_sync(seg, past);
                const long long xf = act ? pos_fx(x) : 0;
                const unsigned slo = __reduce_add_sync(seg, (unsigned)(xf & 0xffffffffll));
                const unsigned shi = __reduce_add_sync(seg, (unsigned)(xf >> 32));
                if (act && lane == __ffs(seg) - 1) {
                    if (sp) atomicAdd(&S.past[li], (int)sp);
                    atomicAdd(&S.psum[li], (unsigned long long)slo + ((unsigned long long)shi << 32));
                }
            }
        }
        __syncthreads();
        if (!obs_only) {
#pragma unroll
            for (int u = 0; u < kPU; ++u)
                if (sidx[u] >= 0) P[sidx[u]] = xn[u];
        }
        __syncthreads();
    }
    if (total == 0) __syncthreads();        // the keys above are complete before they are read
    // ---------------- observation, choice, merge, records ----------------
    unsigned long long *Wt = a.W3 + (size_t)(t % 3) * d.L;
    int4 *Ct = a.crec2 + (size_t)(t & 1) * d.L;
    for (int li = tid; li < nl; li += kPT) {
        const int j = j0 + li;
        const int4 q = S.q[li];
        const int n = q.y;
        int4 stat = S.stat[li];
        if (obs) {
            const int bin = (t - 1) / d.obs_every;
            const size_t o = (size_t)bin * d.L + j;
            const int C = q.w + S.past[li];
            d.out_counts[o] = C - stat.w;
            const longlong2 ps = d.lpos[j];
            const long long pnow = (long long)S.psum[li];
            const long long dist = pnow - ps.x + ps.y;
            d.out_speed[o] = stat.x ? (float)((double)dist / (double)kPosScale / ((double)stat.x * (double)d.dt)) : 0.0f;
            d.out_tt[o] = stat.z ? (float)((double)stat.y * (double)d.dt / (double)stat.z) : 0.0f;
            stat = make_int4(0, 0, 0, C);
            d.lpos[j] = make_longlong2(pnow, 0);
            if (obs_only) { S.stat[li] = stat; continue; }
        }
        stat.x += n;
        S.stat[li] = stat;
        const int4 c0 = S.cr[li];
        const int2 lead = S.lead[li];
        const int4 nd = S.nd[li];
        int tgt = kTgtNone;
        if (c0.x >= 0) {
            if (nd.y == lead.y) {
                tgt = kTgtSink;
            } else {
                tgt = p_choose(d, first, Cp, Wp, S.key[li], S.tv[li], d.loinfo + nd.z, nd.w - nd.z, lead.y, lead.x, t);
                if (tgt >= 0) atomicMax(Wt + tgt, merge_word(S.mkey[li], lead.x));
            }
        }
        const float4 g = S.g[li];
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
        const int4 rec = make_int4(c0.x, c0.x >= 0 ? tgt : kTgtNone, (c0.z << 8) | bits, __float_as_int(x0));
        S.cr[li] = rec;
        Ct[j] = rec;
    }
    for (int ni = tid; ni < nn; ni += kPT) {
        const int2 lead = S.nlead[ni];
        int tgt = kTgtNone;
        if (lead.x >= 0) {
            if (S.nzone[ni] == lead.y) {
                tgt = kTgtSink;
            } else {
                const int4 nq = S.nq[ni];
                tgt = p_choose(d, first, Cp, Wp, S.nkey[ni], S.ntv[ni], d.noinfo + nq.z, nq.w - nq.z, lead.y, lead.x, t);
                if (tgt >= 0) atomicMax(Wt + tgt, merge_word(S.nmkey[ni], lead.x));
            }
        }
        S.nrec[ni] = make_int2(lead.x, tgt);
    }
}

__global__ void __launch_bounds__(kPT, 1) k_persist(DevSim d, PArgs a) {
    extern __shared__ __align__(16) unsigned char p_smem[];
    PSmem &S = *reinterpret_cast<PSmem *>(p_smem);
    float *P = reinterpret_cast<float *>(p_smem + sizeof(PSmem));
    const int tid = threadIdx.x;
    const int j0 = a.grp_links[blockIdx.x];
    const int nl = a.grp_links[blockIdx.x + 1] - j0;
    const int n0 = blockIdx.x * a.npg;
    const int nn = max(0, min(a.npg, d.V - n0));
    const int base0 = nl > 0 ? d.lst[j0].x : 0;
    const int nslots = nl > 0 ? d.lst[j0 + nl - 1].x + d.lst[j0 + nl - 1].y - base0 : 0;
    // ---------------- load the group's state ----------------
    for (int li = tid; li < nl; li += kPT) {
        const int j = j0 + li;
        S.q[li] = d.lq[j];
        S.st[li] = d.lst[j];
        S.g[li] = d.geo[j];
        S.nd[li] = d.lnode[j];
        S.stat[li] = d.lstat[j];
        S.flags[li] = d.vac[j];
        S.cr[li] = d.crec[j];
    }
    for (int ni = tid; ni < nn; ni += kPT) {
        const int n = n0 + ni;
        S.nq[ni] = make_int4(d.fifo_ptr[n], d.fifo_end[n], d.no_ptr[n], d.no_ptr[n + 1]);
        S.nzone[ni] = d.node_zone[n];
        S.nrec[ni] = d.nrec[n];
    }
    const float *pc = (a.t0 & 1) ? d.pos1 : d.pos0;
    for (int s = tid; s < nslots; s += kPT) P[s] = pc[base0 + s];
    if (tid < 4) S.cnt[tid] = 0;
    if (tid == 0) S.stop = 0;
    __syncthreads();
    // ---------------- steps ----------------
    unsigned epoch = 0;
    for (int t = a.t0; t < a.t1; ++t) {
        if (t > a.t0) {
            p_transfers(d, a, S, P, j0, nl, nn, base0, t - 1);
            __syncthreads();
        }
        p_step(d, a, S, P, j0, nl, n0, nn, base0, t, t == a.t0, false);
        ++epoch;
        if (!grid_sync(d, a.bar, epoch * gridDim.x, t, &S.stop)) return;
    }
    if (a.t1 > a.t0) {
        p_transfers(d, a, S, P, j0, nl, nn, base0, a.t1 - 1);
        __syncthreads();
    }
    if (a.final_obs) {
        p_step(d, a, S, P, j0, nl, n0, nn, base0, a.t1, a.t1 == a.t0, true);
        __syncthreads();
    }
    // ---------------- write the group's state back ----------------
    // merge words as the two-kernel executor leaves them: those of the last
    // step in its parity buffer (read by sim_get_records), the other buffer zero
    float *pd = (a.t1 & 1) ? d.pos1 : d.pos0;
    for (int s = tid; s < nslots; s += kPT) pd[base0 + s] = P[s];
    const unsigned long long *Wl = a.W3 + (size_t)((a.t1 + 2) % 3) * d.L;
    unsigned long long *Wlast = (a.t1 & 1) ? d.W0 : d.W1;
    unsigned long long *Wnext = (a.t1 & 1) ? d.W1 : d.W0;
    for (int li = tid; li < nl; li += kPT) {
        const int j = j0 + li;
        d.lq[j] = S.q[li];
        d.lstat[j] = S.stat[li];
        d.vac[j] = S.flags[li];
        d.crec[j] = S.cr[li];
        if (a.t1 > a.t0) Wlast[j] = __ldcg(Wl + j);
        Wnext[j] = 0ull;
    }
    for (int ni = tid; ni < nn; ni += kPT) {
        const int n = n0 + ni;
        d.fifo_ptr[n] = S.nq[ni].x;
        d.nrec[n] = S.nrec[ni];
    }
}

}  // namespace ts
