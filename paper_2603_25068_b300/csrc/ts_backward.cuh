// Reverse-mode kernels of the simulator (sm_103a).
//
// The derivative is that of the straight-through / trajectory-grafting surrogate
// the method differentiates (Methods "Optimization": jax.grad of the dense
// formulation of SI-A Alg. S1 and SI-B Alg. S2): every discrete decision of the
// recorded rollout is frozen and stop_gradient(v) is the recorded value.  The
// adjoint of the dense state X[i, j] is represented by
//   A[s]              adjoint of the valid entry of the vehicle in queue slot s
//                     (a vehicle on a link keeps its slot from step to step, so
//                     the car-following reads and writes it in place, in slot
//                     order);
//   xbar[i]           adjoint of waiting vehicle i's valid entry (its origin
//                     queue, a virtual inflow link of length 0);
//   eadj[i, r]        adjoint of X[i, m_r] right after vehicle i's r-th entry; an
//                     invalid slot is the identity through time, so its adjoint at
//                     an earlier time is that of the next entry into the link.
// A transfer at step t moves a vehicle from its source (the head slot of a
// link, or an origin queue) to the tail slot of its target: its adjoint at
// t + 1 is read there (grafting passes it on unchanged to the source).
// Per step t, in reverse (a segment of K steps is first recomputed from its
// checkpoint, recording the tape that these kernels read):
//   k_bwd_obs     observation at t + 1 (SI-D): dC_j/dx_i = s sigma (1 - sigma),
//                 s = 5/L_j; demand weight 1 + (lambda - sg lambda)/lambda;
//   k_bwd_node_z  per merge candidate: abar = M (Ebar - Xbar_old) - x Xbar_old
//                 (SI-B Eq. transfer) and its merge-softmax weight; per-target
//                 sums, kept per step of the segment; the winners' entry
//                 adjoints; demand weight of exits;
//   k_bwd_node_g  merge softmax Jacobian -> alpha, lbar; link-choice softmax
//                 Jacobian (Eqs. gumbel, straigththrough) -> U = beta/c + w.phi,
//                 G = w.psi.  Nothing later in the reverse chain reads what it
//                 writes (parameter accumulators only), so it runs once per
//                 segment over all of the segment's steps, beside the chain;
//   k_bwd_cf      car-following (SI-A) by branch tag: free x' = x + u dt,
//                 congested x' = x_leader - dn/kappa, stopped x' = x; the TG clip
//                 passes the adjoint; the winner's old entry receives its new
//                 entry's adjoint unchanged (grafting, SI-C).
// Precision.  FP64 arithmetic runs at a small fraction of the FP32 rate on this
// part, so the kernels do none on the per-vehicle path.  Adjoints whose
// differences cancel (A, xbar, eadj, abar, the merge sums SA / Z and the bin
// adjoints Cbar) are double-float pairs, hi + lo with |lo| <= ulp(hi) / 2
// (about 48 significant bits), computed with FP32 operations through the
// error-free transformations TwoSum (Knuth), FastTwoSum (Dekker) and the
// FMA-based TwoProduct.  Exponentials, softmax weights and per-link sums are
// FP32.  The parameter accumulators are double, updated by atomics that
// execute in L2; only those updates convert to double.
#pragma once
#include "ts_step.cuh"

namespace ts {

// ---- double-float arithmetic (value = x + y of a float2) ----
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {      // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float2 s = ff_two_sum(a.x, b.x);
    const float2 t = ff_two_sum(a.y, b.y);
    s = ff_fast_two_sum(s.x, __fadd_rn(s.y, t.x));
    return ff_fast_two_sum(s.x, __fadd_rn(s.y, t.y));
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    const float e = __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -p));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_div(float2 a, float2 b) {
    const float q1 = __fdiv_rn(a.x, b.x);
    const float2 r = ff_sub(a, ff_mul_f(b, q1));
    return ff_fast_two_sum(q1, __fdiv_rn(r.x, b.x));
}
__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 ff_from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

struct BwdDev {
    int S, K, cap, n_od;
    float tau, inv_tau;
    // tape of the current segment: K steps, K + 1 state records
    float *tpos;                 // [(K+1) S] positions at the start of each step (written at
                                 // bin ends only, where the observation's adjoint reads them)
    int *tvid;                   // [S] vehicle of each occupied slot at the segment start
    int *tent;                   // [L K] entrant log: entrant m of link j in the segment at j K + m
    int4 *tlq;                   // [(K+1) L] queue state at the start of each step
    int8_t *ttag;                // [K S]     car-following tags
    int4 *tcrec;                 // [K L]     link candidates
    int2 *tnrec;                 // [K V]     origin-queue candidates
    unsigned long long *tW;      // [K L]     merge words
    float *tmkey;                // [K (L+V)] merge key of each candidate with a target
    // adjoints (float2 = double-float)
    float2 *A;                   // [S] adjoint of each occupied queue slot
    float2 *xbar;                // [N] adjoint of each waiting vehicle
    float2 *eadj;                // [N cap]
    const int2 *route_log;       // [N cap]
    const int *route_len;        // [N]
    int *cursor;                 // [N] index of each vehicle's latest entry at a step <= t
                                 // (the reverse pass undoes entries from the last one)
    unsigned char *rdup;         // [N] bit 0: the vehicle's route enters some link twice; bit 1: some
                                 // node is the head of two of its links (implied by bit 0)
    const float2 *Cbar;          // [n_bins L] adjoint of C_j at the end of each bin
    const float2 *Csuf;          // [(n_bins + 1) L] suffix sums of Cbar
    double *gu, *gs, *ga, *gU, *gG;   // [L]
    double *gao;                 // [1]
    double *glam;                // [n_od]
    // per tape set, by tape record (step t0 + rec of the segment):
    double *Z, *SA;              // [K L] per-target merge sums (zero before the segment)
    float *ebuf;                 // [K (L + V)] per-source merge weight
    float2 *abuf;                // [K (L + V)] per-source abar
    const int *od;               // [N]
    const float *od_lambda;      // [n_od]
};

__device__ __forceinline__ float merge_key_of(unsigned long long w) {
    const uint32_t o = (uint32_t)(w >> 32);
    const uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(b);
}

// First index k in [k0, n) of vehicle v's route log whose entry (step, link)
// satisfies pred, or -1.  Entries are read eight at a time with independent
// 16-byte loads (rows are 64-byte aligned: the capacity is a multiple of 8).
// A row holds cap entries, so each batch is loaded before the entry count is
// known (the first batch's loads overlap that of the count); entries past the
// count are ignored.
template <class Pred>
__device__ __forceinline__ int route_find(const BwdDev &b, int v, int k0, Pred pred) {
    const int n = b.route_len[v];
    const int4 *r = reinterpret_cast<const int4 *>(b.route_log + (size_t)v * b.cap);
    for (int base = k0 & ~7; base < b.cap; base += 8) {
        int4 w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = r[(base >> 1) + q];
        if (base >= n) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ka = base + 2 * q, kb = ka + 1;
            if (ka >= k0 && ka < n && pred(w[q].x, w[q].y)) return ka;
            if (kb >= k0 && kb < n && pred(w[q].z, w[q].w)) return kb;
        }
    }
    return -1;
}

// Per vehicle (a warp each): the reverse pass's entry cursor starts at the last
// entry; whether the route enters some link twice, and whether some node is the
// head of two of its links (values compared within 32-entry chunks by match,
// across chunks by shuffles).  A link entered twice has its head twice, so the
// search ends at the first repeated link.
__global__ void k_route_scan(DevSim d, int N, BwdDev b) {
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (v >= N) return;
    const int n = b.route_len[v];
    const int2 *r = b.route_log + (size_t)v * b.cap;
    bool dup = false, hdup = false;
    for (int a = 0; a < n && !dup; a += 32) {
        const int la = a + lane < n ? r[a + lane].y : -1;
        const int xa = la >= 0 ? la : -1 - lane;                          // padding never matches
        const int ha = la >= 0 ? d.lnode[la].x : -1 - lane;
        const unsigned mx = __match_any_sync(kFull, xa), mh = __match_any_sync(kFull, ha);   // every lane
        dup = __any_sync(kFull, xa >= 0 && __popc(mx) > 1);
        hdup = hdup || __any_sync(kFull, ha >= 0 && __popc(mh) > 1);
        for (int c = a + 32; c < n && !dup; c += 32) {
            const int lc = c + lane < n ? r[c + lane].y : -1;
            const int xc = lc >= 0 ? lc : -1000 - lane;
            const int hc = lc >= 0 ? d.lnode[lc].x : -1000 - lane;
            bool hit = false, hhit = false;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                hit |= xa == __shfl_sync(kFull, xc, q);
                hhit |= ha == __shfl_sync(kFull, hc, q);
            }
            dup = __any_sync(kFull, hit);
            hdup = hdup || __any_sync(kFull, hhit);
        }
    }
    if (lane == 0) {
        b.cursor[v] = n - 1;
        b.rdup[v] = (dup ? 1 : 0) | ((dup || hdup) ? 2 : 0);
    }
}

// copy the state at the start of step (t0 + rec) into the tape (positions and
// queue states; the vehicles follow from the entrant log)
__global__ void k_tape_pre(DevSim d, BwdDev b, int rec, int cur) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float *pc = cur ? d.pos1 : d.pos0;
    if (i < b.S) b.tpos[(size_t)rec * b.S + i] = pc[i];
    if (i < d.L) b.tlq[(size_t)rec * d.L + i] = d.lq[i];
}

// Vehicle with entry index e of link j (e = exits so far + queue position; a
// link takes its entrants in FIFO order): one that was queued at the segment
// start (queue state q0: ring slot from the start record of the tape), else
// entrant e - (q0.w + q0.y) of the segment's entrant log.
__device__ __forceinline__ int vid_at(const BwdDev &b, int j, int4 q0, int base, int cap, int e) {
    const int m = e - (q0.w + q0.y);
    if (m >= 0) return b.tent[(size_t)j * b.K + m];
    int idx = q0.x + (e - q0.w);
    if (idx >= cap) idx -= cap;
    return b.tvid[base + idx];
}

// adjoints at the end of the rollout: dL/dx(T) for the vehicles on links (in
// their slots, one warp per link of the final state), zero for waiting ones
__global__ void k_bwd_init(DevSim d, BwdDev b, const float *dxT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.N) b.xbar[i] = make_float2(0.0f, 0.0f);
    const int j = i >> 5, lane = threadIdx.x & 31;
    if (j >= d.L) return;
    const int4 q = d.lq[j], st = d.lst[j];
    for (int k = lane; k < q.y; k += 32) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        b.A[st.x + idx] = make_float2(dxT ? dxT[d.saux[st.x + idx].x] : 0.0f, 0.0f);
    }
}

// (1) observation at time t + 1 = the state of tape record rec: one warp per link.
// dC/dx = s sigma(z) (1 - sigma(z)), z = s (x - L / 2), in the form
// s a / (1 + a)^2 with a = exp(-|z|) (symmetric in z, no cancellation).
__global__ void k_bwd_obs(DevSim d, BwdDev b, int rec, int bin) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= d.L) return;
    const float2 cb = b.Cbar[(size_t)bin * d.L + j];
    if (cb.x == 0.0f) return;
    const int4 q = b.tlq[(size_t)rec * d.L + j], q0 = b.tlq[j];
    const int4 st = d.lst[j];
    const float len = d.geo[j].x, s5 = __fdiv_rn(5.0f, len), half = __fmul_rn(0.5f, len);
    for (int k = lane; k < q.y; k += 32) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        const size_t o = (size_t)rec * b.S + st.x + idx;
        const float x = b.tpos[o];
        const float a = expf(-fabsf(__fmul_rn(s5, __fsub_rn(x, half))));
        const float a1 = __fadd_rn(1.0f, a);
        const float w = __fdiv_rn(__fmul_rn(s5, a), __fmul_rn(a1, a1));
        b.A[st.x + idx] = ff_add(b.A[st.x + idx], ff_mul_f(cb, w));
        if (x >= half) {
            const int k2 = b.od[vid_at(b, j, q0, st.x, st.y, q.w + k)];
            atomicAdd(&b.glam[k2], (double)__fdiv_rn(cb.x, b.od_lambda[k2]));
        }
    }
}

struct Cand {
    int vid, tgt, src;        // src: link id, or L + node
    float x, alpha;
    bool won;
};

__device__ __forceinline__ Cand load_cand(const DevSim &d, const BwdDev &b, int i, int rec) {
    Cand c;
    const unsigned long long *W = b.tW + (size_t)rec * d.L;
    if (i < d.L) {
        const int4 r = b.tcrec[(size_t)rec * d.L + i];
        c.vid = r.x; c.tgt = r.y; c.x = __int_as_float(r.w); c.alpha = d.alpha[i];
    } else {
        const int2 r = b.tnrec[(size_t)rec * d.V + (i - d.L)];
        c.vid = r.x; c.tgt = r.y; c.x = 0.0f; c.alpha = d.alpha[d.L];
    }
    c.src = i;
    c.won = c.vid >= 0 && c.tgt >= 0 && W[c.tgt] != 0ull && merge_vid(W[c.tgt]) == c.vid;
    return c;
}

// (2a) merge candidate i of step t (link, or L + origin node): abar, merge-
// softmax weight, per-target sums (by tape record), the winner's entry
// adjoint and cursor, the demand weight of exits.  z_load issues the record,
// then in one round the target's merge word and everything that depends on the
// vehicle only (its adjoint at t + 1 among them); z_finish does the rest.
struct ZLoad {
    float2 xv;                   // the vehicle's adjoint at t + 1
    unsigned long long wt;       // the target's merge word
    int v, tgt, cur, dup, k2;
    int aslot;                   // slot holding that adjoint (target's tail if the vehicle
                                 // entered it, else the source's head), -1: waiting (xbar)
    bool won;
    float x, csuf, key;          // key: the candidate's merge key alpha + g' (recorded)
};

// Programmatic dependent launch: the next kernel of the stream may start
// (and issue its loads of the tape and of static data) while this one runs;
// pdl_wait returns once the previous kernel has completed and its writes are
// visible, and comes before any access to what that kernel writes.  In a
// kernel launched without the attribute it returns at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// z_load: the record and what depends on the tape or static data only;
// z_load_adj: the adjoint state the previous step wrote (after pdl_wait)
__device__ __forceinline__ bool z_load(const DevSim &d, const BwdDev &b, int i, int rec, int bin0, ZLoad &z) {
    if (i < d.L) {
        const int4 r = b.tcrec[(size_t)rec * d.L + i];
        z.v = r.x; z.tgt = r.y; z.x = __int_as_float(r.w);
    } else {
        const int2 r = b.tnrec[(size_t)rec * d.V + (i - d.L)];
        z.v = r.x; z.tgt = r.y; z.x = 0.0f;
    }
    if (z.v < 0) return false;
    z.wt = z.tgt >= 0 ? b.tW[(size_t)rec * d.L + z.tgt] : 0ull;
    z.key = z.tgt >= 0 ? b.tmkey[(size_t)rec * (d.L + d.V) + i] : 0.0f;
    z.won = z.tgt >= 0 && z.wt != 0ull && merge_vid(z.wt) == z.v;
    z.aslot = -1;
    if (z.won) {                 // the entrant is the last vehicle of the target's queue at t + 1
        const int4 qm = b.tlq[(size_t)(rec + 1) * d.L + z.tgt], stm = d.lst[z.tgt];
        int idx = qm.x + qm.y - 1;
        if (idx >= stm.y) idx -= stm.y;
        z.aslot = stm.x + idx;
    } else if (i < d.L) {        // still the leader of link i
        z.aslot = d.lst[i].x + b.tlq[(size_t)rec * d.L + i].x;
    }
    z.dup = b.rdup[z.v];
    z.k2 = b.od[z.v];
    z.csuf = i < d.L ? b.Csuf[(size_t)bin0 * d.L + i].x : 0.0f;
    return true;
}
__device__ __forceinline__ void z_load_adj(const BwdDev &b, ZLoad &z) {
    z.cur = b.cursor[z.v];
    z.xv = z.aslot >= 0 ? b.A[z.aslot] : b.xbar[z.v];
}

__device__ __forceinline__ void z_finish(const DevSim &d, const BwdDev &b, int i, int t, int rec, const ZLoad &z) {
    const int v = z.v, tgt = z.tgt, cur = z.cur;
    const bool won = z.won;
    const bool exits = i < d.L && (won || tgt == kTgtSink);         // an exit from link i
    const float lam = exits ? b.od_lambda[z.k2] : 1.0f;
    if (won) {                   // adjoint right after this entry: the latest one not yet undone
        b.cursor[v] = cur - 1;
        if (cur >= 0) b.eadj[(size_t)v * b.cap + cur] = z.xv;
        if (i >= d.L) b.xbar[v] = z.xv;                  // a waiting vehicle before its entry (grafting)
    }
    if (tgt >= 0) {
        // (alpha + g') is the merge key of the forward step (recorded); the
        // largest key of the target is in its merge word
        const float e = expf(__fmul_rn(__fsub_rn(z.key, merge_key_of(z.wt)), b.inv_tau));
        float2 Enew, Xold;
        if (won) {
            Enew = z.xv;
            Xold = make_float2(0.0f, 0.0f);
            if (i < d.L && cur >= 0 && (z.dup & 1)) {            // next re-entry into the source link
                const int k = route_find(b, v, cur + 1, [&](int, int l) { return l == i; });
                if (k >= 0) Xold = b.eadj[(size_t)v * b.cap + k];
            }
        } else {                 // first entry into the target after the current one
            Enew = make_float2(0.0f, 0.0f);
            int k = -1;
            if (i < d.L && !(z.dup & 2)) {
                // the target starts at the head of link i (entry cur); an entry into it
                // past cur + 1 would make that node the head of a second link of the route
                if (cur + 1 < b.route_len[v]) {
                    const int2 e = b.route_log[(size_t)v * b.cap + cur + 1];
                    if (e.x > t && e.y == tgt) k = cur + 1;
                }
            } else {
                k = route_find(b, v, cur + 1, [&](int s, int l) { return s > t && l == tgt; });
            }
            if (k >= 0) Enew = b.eadj[(size_t)v * b.cap + k];
            Xold = z.xv;
        }
        const float2 abar = ff_sub(ff_mul_f(ff_sub(Enew, Xold), d.M), ff_mul_f(Xold, z.x));
        const size_t eo = (size_t)rec * (d.L + d.V) + i;
        b.ebuf[eo] = e;
        b.abuf[eo] = abar;
        const size_t zo = (size_t)rec * d.L + tgt;
        atomicAdd(&b.Z[zo], (double)e);
        atomicAdd(&b.SA[zo], ff_to_double(ff_mul_f(abar, e)));
    }
    if (exits) atomicAdd(&b.glam[z.k2], (double)__fdiv_rn(z.csuf, lam));
}

// (2b) merge and link-choice Jacobians of steps t0 .. t0 + nrec - 1 (tape
// records 0 .. nrec - 1), one thread per (record, candidate)
__global__ void k_bwd_node_g(DevSim d, BwdDev b, int t0, int nrec) {
    const int LV = d.L + d.V;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)nrec * LV) return;
    const int rec = (int)(g / LV), i = (int)(g - (long long)rec * LV), t = t0 + rec;
    const Cand c = load_cand(d, b, i, rec);
    if (c.vid < 0 || c.tgt < 0) return;
    const size_t zo = (size_t)rec * d.L + c.tgt;
    const float2 Z = ff_from_double(b.Z[zo]);
    const float2 S = ff_div(ff_from_double(b.SA[zo]), Z);            // softmax-weighted mean of abar
    const size_t eo = (size_t)rec * LV + i;
    const float pi = __fdiv_rn(b.ebuf[eo], Z.x);
    const float vbar = __fmul_rn(__fmul_rn(pi, ff_sub(b.abuf[eo], S).x), b.inv_tau);   // adjoint of V'_i
    if (i < d.L) atomicAdd(&b.ga[i], (double)vbar); else atomicAdd(b.gao, (double)vbar);
    const float lbar = __fmul_rn(c.alpha, vbar);                     // adjoint of l_i at the target
    if (lbar == 0.0f) return;
    // choice set of the candidate
    const int v = c.vid;
    const int zone = d.dest_zone[v];
    const float4 *info;
    int deg;
    if (i < d.L) {
        const int4 nd = d.lnode[i];
        info = d.loinfo + nd.z;
        deg = nd.w - nd.z;
    } else {
        const int n = i - d.L;
        info = d.noinfo + d.no_ptr[n];
        deg = d.no_ptr[n + 1] - d.no_ptr[n];
    }
    // the forward step's choice keys V_k + g_k of the first kG slots held in
    // registers (fully unrolled); slots past kG are recomputed where needed.
    // Softmax weights exp((key_k - key_max) / tau).
    constexpr int kG = 8;
    auto keyk = [&](int k, int &m, float &df) {
        const float4 e = info[k];
        m = __float_as_int(e.w);
        df = d.dest_feat[(size_t)zone * d.V + __float_as_int(e.z)];
        const float util = __fadd_rn(e.x, __fmul_rn(e.y, df));
        return __fadd_rn(util, gumbel(d.key0, d.key1, v, t, 0, k));
    };
    const float itau = b.inv_tau;
    float key[kG], dfs[kG];
    int ms[kG];
    float kmax = -INFINITY;
    int ks = 0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            key[k] = keyk(k, ms[k], dfs[k]);
            kmax = fmaxf(kmax, key[k]);
            if (ms[k] == c.tgt) ks = k;
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const float kk = keyk(k, m, df);
        kmax = fmaxf(kmax, kk);
        if (m == c.tgt) ks = k;
    }
    float zs = 0.0f, eks = 0.0f;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            key[k] = expf(__fmul_rn(__fsub_rn(key[k], kmax), itau));
            zs = __fadd_rn(zs, key[k]);
            if (k == ks) eks = key[k];
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const float ek = expf(__fmul_rn(__fsub_rn(keyk(k, m, df), kmax), itau));
        zs = __fadd_rn(zs, ek);
        if (k == ks) eks = ek;
    }
    const float pks = __fdiv_rn(eks, zs);
    const float lt = __fmul_rn(lbar, itau);
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            const float pk = __fdiv_rn(key[k], zs);
            const float Vbar = __fmul_rn(__fmul_rn(pk, __fsub_rn(k == ks ? 1.0f : 0.0f, pks)), lt);
            atomicAdd(&b.gU[ms[k]], (double)Vbar);
            atomicAdd(&b.gG[ms[k]], (double)__fmul_rn(Vbar, dfs[k]));
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const float pk = __fdiv_rn(expf(__fmul_rn(__fsub_rn(keyk(k, m, df), kmax), itau)), zs);
        const float Vbar = __fmul_rn(__fmul_rn(pk, __fsub_rn(k == ks ? 1.0f : 0.0f, pks)), lt);
        atomicAdd(&b.gU[m], (double)Vbar);
        atomicAdd(&b.gG[m], (double)__fmul_rn(Vbar, df));
    }
}

// (2a + 3) merge adjoint and car-following of step (t0 + rec), one launch.
// A block takes kCfLinks consecutive links and npb origin queues:
//   * car-following warps: each thread takes kCfE consecutive positions of the
//     links' concatenated queues (leader first), so that every tape and
//     adjoint load of a pass is in flight at once.  Vehicle k's adjoint at
//     time t is its own adjoint at t + 1 unless its update was congested (then
//     x' depended on the leader only), plus its follower's adjoint when the
//     follower was congested (the follower's headway used x_k).  The
//     follower's values come from the same thread, from the next thread
//     (shared memory) or, for the last position of a pass, from a look-ahead
//     load.  The per-link parameter sums (free -> u: x' = x + u dt, congested
//     -> s) are reduced in a fixed order.  These warps synchronise among
//     themselves with a named barrier.
//   * merge warps: one thread per link candidate and per origin-queue
//     candidate (z_load, z_finish).
// A link's candidate is its leader, whose adjoint car-following overwrites, so
// the two groups meet once, at a block barrier before the first write: by then
// every candidate's adjoint at t + 1 has been read.  The merge warps then
// finish their route-log chains while car-following computes and writes.
constexpr int kCfWarps = 5, kZWarps = 3;
constexpr int kCfThreads = 32 * kCfWarps;
constexpr int kBwdThreads = 32 * (kCfWarps + kZWarps);
constexpr int kCfLinks = 64;
constexpr int kZNodeThreads = 32 * kZWarps - kCfLinks;
constexpr int kCfE = 8;
constexpr int kCfPass = kCfThreads * kCfE;

__device__ __forceinline__ void cf_bar() { asm volatile("bar.sync 1, %0;" :: "n"(kCfThreads) : "memory"); }

__global__ void __launch_bounds__(kBwdThreads, 4) k_bwd_step(DevSim d, BwdDev b, int rec, int t, int bin0, int npb) {
    __shared__ int4 sq[kCfLinks];
    __shared__ int sbase[kCfLinks], scap[kCfLinks], off[kCfLinks + 1];
    __shared__ int sld[kCfLinks];                       // leader's transfer: 0 none / lost, 1 entered a link, 2 arrived
    __shared__ float2 sen[kCfLinks];                    // adjoint at t + 1 of a leader that entered a link
    __shared__ int ftag[kCfThreads];
    __shared__ float2 fg[kCfThreads];
    __shared__ int skf[kCfThreads], skl[kCfThreads];   // link of each thread's first / last run of the pass
    __shared__ float2 spl[kCfThreads];                  // sums of each thread's last run
    __shared__ float lsu[kCfLinks], lss[kCfLinks];
    const int tid = threadIdx.x, lane = tid & 31;
    const int j0 = blockIdx.x * kCfLinks;
    const int nl = min(kCfLinks, d.L - j0);
    pdl_trigger();
    if (tid >= kCfThreads) {                            // merge warps
        // a thread's first candidate (its link, or its first origin queue) is
        // loaded before the block barrier, the rest of its origin queues after
        const int zi = tid - kCfThreads;
        const int n0 = blockIdx.x * npb + zi - kCfLinks, n1 = min(d.V, (blockIdx.x + 1) * npb);
        const int i = zi < nl ? j0 + zi : (zi >= kCfLinks && n0 < n1) ? d.L + n0 : -1;
        ZLoad z;
        const bool has = i >= 0 && z_load(d, b, i, rec, bin0, z);
        pdl_wait();
        if (has) {
            z_load_adj(b, z);
            asm volatile("" :: "f"(z.xv.x), "f"(z.xv.y));   // in before the barrier: car-following
        }                                                      // then rewrites the leader's slot
        if (zi < nl) {                                  // for the car-following of the link's leader
            const int f = has ? (z.won ? 1 : (z.tgt == kTgtSink ? 2 : 0)) : 0;
            sld[zi] = f;
            if (f == 1) sen[zi] = z.xv;
        }
        __syncthreads();
        if (has) z_finish(d, b, i, t, rec, z);
        if (zi >= kCfLinks) {                           // origin queues (not touched by car-following)
            for (int n = n0 + kZNodeThreads; n < n1; n += kZNodeThreads) {
                ZLoad zn;
                if (z_load(d, b, d.L + n, rec, bin0, zn)) {
                    z_load_adj(b, zn);
                    z_finish(d, b, d.L + n, t, rec, zn);
                }
            }
        }
        return;
    }
    if (tid < kCfLinks) {                               // queue states of the block's links
        if (tid < nl) {
            const int j = j0 + tid;
            const int4 q = b.tlq[(size_t)rec * d.L + j];
            const int4 st = d.lst[j];
            sq[tid] = q;
            sbase[tid] = st.x;
            scap[tid] = st.y;
        }
        lsu[tid] = 0.0f;
        lss[tid] = 0.0f;
    }
    cf_bar();
    if (tid < 32) {                                     // exclusive scan of the queue lengths (warp 0)
        const int a = tid < nl ? sq[tid].y : 0, c = tid + 32 < nl ? sq[tid + 32].y : 0;
        int ia = a, ic = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(kFull, ia, o), yc = __shfl_up_sync(kFull, ic, o);
            if (lane >= o) { ia += ya; ic += yc; }
        }
        const int ta = __shfl_sync(kFull, ia, 31);
        off[tid] = ia - a;
        off[tid + 32] = ta + ic - c;
        if (tid == 31) off[kCfLinks] = ta + ic;
    }
    cf_bar();
    const int total = off[kCfLinks];
    const float dt = d.dt;
    const int8_t *ttag = b.ttag + (size_t)rec * b.S;
    auto slot_of = [&](int li, int e) {
        int idx = sq[li].x + (e - off[li]);
        if (idx >= scap[li]) idx -= scap[li];
        return sbase[li] + idx;
    };
    bool met = false;                                   // the block barrier with the merge warps
    for (int base = 0; base < total; base += kCfPass) {
        const int e0 = base + tid * kCfE;
        int sl[kCfE], tag[kCfE], lk[kCfE];
        float2 g[kCfE];
        int li = e0 < total ? link_of(off, nl, e0) : 0;
#pragma unroll
        for (int u = 0; u < kCfE; ++u) {
            const int e = e0 + u;
            sl[u] = -1;
            tag[u] = kTagStop;
            lk[u] = 0;
            if (e < total) {
                li = link_advance(off, nl, li, e);
                lk[u] = li;
                sl[u] = slot_of(li, e);
                tag[u] = ttag[sl[u]];
            }
        }
        int sx = -1, tx = kTagStop;                     // the position after this pass
        const int ex = base + kCfPass;
        if (tid == kCfThreads - 1 && ex < total) {
            sx = slot_of(link_of(off, nl, ex), ex);
            tx = ttag[sx];
        }
        pdl_wait();                                     // adjoints of the previous step from here on
#pragma unroll
        for (int u = 0; u < kCfE; ++u) g[u] = sl[u] >= 0 ? b.A[sl[u]] : make_float2(0.0f, 0.0f);
        const float2 gx = sx >= 0 ? b.A[sx] : make_float2(0.0f, 0.0f);
        ftag[tid] = tag[0];
        fg[tid] = g[0];
        if (!met) {
            __syncthreads();
            met = true;
        } else {
            cf_bar();
        }
        const int ntag = tid + 1 < kCfThreads ? ftag[tid + 1] : tx;
        const float2 ng = tid + 1 < kCfThreads ? fg[tid + 1] : gx;
        // a leader that left its link at t: its adjoint at t + 1 is in its
        // target's slot (entered, from the merge warps) or zero (arrived).  A
        // leader is nobody's follower, so fg / ng need no such change.
#pragma unroll
        for (int u = 0; u < kCfE; ++u) {
            if (e0 + u < total && e0 + u == off[lk[u]]) {
                const int f = sld[lk[u]];
                if (f == 1) g[u] = sen[lk[u]];
                else if (f == 2) g[u] = make_float2(0.0f, 0.0f);
            }
        }
        // adjoints at time t, and the per-link parameter sums of the pass
        // (free -> u, congested -> s): a run of one link's positions inside
        // this thread is summed here, in order; a link whose positions span
        // several threads is finished by the thread that holds its last
        // position of the pass, which adds the last runs of the threads before
        // it, right to left (a fixed order)
        float su = 0.0f, ss = 0.0f, fu = 0.0f, fs = 0.0f;
        int rl = -1, kf = -1;
#pragma unroll
        for (int u = 0; u < kCfE; ++u) {
            const int e = e0 + u;
            if (e >= total) break;
            const int ft = u + 1 < kCfE ? tag[u + 1 < kCfE ? u + 1 : u] : ntag;
            const float2 fv = u + 1 < kCfE ? g[u + 1 < kCfE ? u + 1 : u] : ng;
            const bool own = tag[u] != kTagCong, fol = e + 1 < off[lk[u] + 1] && ft == kTagCong;
            const float2 pre = own ? (fol ? ff_add(g[u], fv) : g[u]) : (fol ? fv : make_float2(0.0f, 0.0f));
            b.A[sl[u]] = pre;
            if (lk[u] != rl) {                          // a new run; close the previous one
                if (rl >= 0) {
                    if (kf < 0) { kf = rl; fu = su; fs = ss; }      // the first run
                    else { lsu[rl] += su; lss[rl] += ss; }          // a whole link inside this thread
                }
                rl = lk[u];
                su = 0.0f;
                ss = 0.0f;
            }
            su = __fadd_rn(su, (tag[u] == kTagFree) ? __fmul_rn(g[u].x, dt) : 0.0f);
            ss = __fadd_rn(ss, (tag[u] == kTagCong) ? -g[u].x : 0.0f);
        }
        const bool single = kf < 0;                     // one run only: it is both the first and the last
        if (single) { kf = rl; fu = su; fs = ss; }
        skf[tid] = kf;
        skl[tid] = rl;
        spl[tid] = make_float2(su, ss);
        cf_bar();
        const int nf = tid + 1 < kCfThreads ? skf[tid + 1] : -1;
        if (kf >= 0 && (!single || nf != kf)) {         // the first run ends the link's positions here
            float tu = fu, ts = fs;
            for (int j = tid - 1; j >= 0 && skl[j] == kf; --j) {
                const float2 p = spl[j];
                tu = __fadd_rn(tu, p.x);
                ts = __fadd_rn(ts, p.y);
                if (skf[j] != kf) break;                // thread j's last run starts inside it
            }
            lsu[kf] += tu;
            lss[kf] += ts;
        }
        if (!single && nf != rl) {                      // the last run ends the link here too
            lsu[rl] += su;
            lss[rl] += ss;
        }
        cf_bar();                                       // before the next pass reuses the buffers
    }
    if (!met) __syncthreads();                          // no vehicles: meet the merge warps anyway
    pdl_wait();
    if (tid < nl) {
        if (lsu[tid] != 0.0f) b.gu[j0 + tid] += (double)lsu[tid];
        if (lss[tid] != 0.0f) b.gs[j0 + tid] += (double)lss[tid];
    }
}

// per-feature partial sums of dL/dw = sum_l gU_l phi_lf + gG_l psi_lf over the
// 256 links of a block, in a fixed tree order (deterministic)
constexpr int kGwLinks = 256;
__global__ void __launch_bounds__(kGwLinks) k_bwd_gw_part(DevSim d, BwdDev b, const float *phi, const float *psi,
                                                         double *part) {
    __shared__ double red[kGwLinks];
    const int tid = threadIdx.x, l = blockIdx.x * kGwLinks + tid;
    for (int f = 0; f < d.F; ++f) {
        red[tid] = l < d.L ? b.gU[l] * (double)phi[(size_t)l * d.F + f] + b.gG[l] * (double)psi[(size_t)l * d.F + f]
                           : 0.0;
        __syncthreads();
        for (int st = kGwLinks / 2; st > 0; st >>= 1) {
            if (tid < st) red[tid] += red[tid + st];
            __syncthreads();
        }
        if (tid == 0) part[(size_t)blockIdx.x * d.F + f] = red[0];
        __syncthreads();
    }
}

// parameter gradients from the accumulators: u dt, s = dn / kappa,
// U = beta / c + w.phi, G = w.psi
__global__ void k_bwd_finalize(DevSim d, BwdDev b, const float *kappa, const float *beta, const float *cost,
                               const double *gw_part, int n_part, float dn, float *gu_o, float *gk_o,
                               float *ga_o, float *gb_o, float *gc_o, float *gw_o, float *gao_o, float *gl_o) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < d.L) {
        const double kap = kappa[j], c = cost[j], be = beta[j];
        if (gu_o) gu_o[j] = (float)b.gu[j];
        if (gk_o) gk_o[j] = (float)(b.gs[j] * (-(double)dn / (kap * kap)));
        if (ga_o) ga_o[j] = (float)b.ga[j];
        if (gb_o) gb_o[j] = (float)(b.gU[j] / c);
        if (gc_o) gc_o[j] = (float)(-b.gU[j] * be / (c * c));
    }
    if (j < d.F && gw_o) {
        double s = 0.0;
        for (int p = 0; p < n_part; ++p) s += gw_part[(size_t)p * d.F + j];
        gw_o[j] = (float)s;
    }
    if (j == 0 && gao_o) *gao_o = (float)*b.gao;
    if (j < b.n_od && gl_o) gl_o[j] = (float)b.glam[j];
}

}  // namespace ts
