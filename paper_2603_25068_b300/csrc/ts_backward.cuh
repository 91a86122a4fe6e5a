// Reverse-mode kernels of the simulator (sm_103a).
//
// The derivative is that of the straight-through / trajectory-grafting surrogate
// the method differentiates (Methods "Optimization": jax.grad of the dense
// formulation of SI-A Alg. S1 and SI-B Alg. S2): every discrete decision of the
// recorded rollout is frozen and stop_gradient(v) is the recorded value.  The
// dense state X[i, j] is represented by
//   xbar[i]           adjoint of vehicle i's valid entry (its link, or its origin
//                     queue, a virtual inflow link of length 0), and
//   eadj[i, r]        adjoint of X[i, m_r] right after vehicle i's r-th entry; an
//                     invalid slot is the identity through time, so its adjoint at
//                     an earlier time is that of the next entry into the link.
// Per step t, in reverse (a segment of K steps is first recomputed from its
// checkpoint, recording the tape that these kernels read):
//   k_bwd_obs     observation at t + 1 (SI-D): dC_j/dx_i = s sigma (1 - sigma),
//                 s = 5/L_j; demand weight 1 + (lambda - sg lambda)/lambda;
//   k_bwd_node_z  per merge candidate: abar = M (Ebar - Xbar_old) - x Xbar_old
//                 (SI-B Eq. transfer) and its merge-softmax weight; per-target
//                 sums; the winners' entry adjoints; demand weight of exits;
//   k_bwd_node_g  merge softmax Jacobian -> alpha, lbar; link-choice softmax
//                 Jacobian (Eqs. gumbel, straigththrough) -> U = beta/c + w.phi,
//                 G = w.psi;
//   k_bwd_cf      car-following (SI-A) by branch tag: free x' = x + u dt,
//                 congested x' = x_leader - dn/kappa, stopped x' = x; the TG clip
//                 passes the adjoint; the winner's old entry receives its new
//                 entry's adjoint unchanged (grafting, SI-C).
// Accumulators are double precision.
#pragma once
#include "ts_step.cuh"

namespace ts {

struct BwdDev {
    int S, K, cap, n_od;
    float tau, inv_tau;
    // tape of the current segment: K steps, K + 1 state records
    float *tpos;                 // [(K+1) S] positions at the start of each step
    int *tvid;                   // [(K+1) S] vehicle of each slot
    int4 *tlq;                   // [(K+1) L] queue state at the start of each step
    int8_t *ttag;                // [K S]     car-following tags
    int4 *tcrec;                 // [K L]     link candidates
    int2 *tnrec;                 // [K V]     origin-queue candidates
    unsigned long long *tW;      // [K L]     merge words
    // adjoints
    double *xbar;                // [N]
    double *eadj;                // [N cap]
    const int2 *route_log;       // [N cap]
    const int *route_len;        // [N]
    const double *Cbar;          // [n_bins L] adjoint of C_j at the end of each bin
    const double *Csuf;          // [(n_bins + 1) L] suffix sums of Cbar
    double *gu, *gs, *ga, *gU, *gG;   // [L]
    double *gao;                 // [1]
    double *glam;                // [n_od]
    double *Z, *SA;              // [2 L] per-target merge sums, by step parity (the
                                 // reverse car-following kernel clears the other parity)
    double *ebuf, *abuf;         // [2 (L + V)] per-source merge weight and abar, by step
                                 // parity (the Jacobian kernel of step t runs beside
                                 // the merge kernel of step t - 1)
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

// adjoint right after vehicle v's first entry into link m at a step > t (0 if none)
__device__ __forceinline__ double next_entry(const BwdDev &b, int v, int m, int t) {
    const int k = route_find(b, v, 0, [&](int s, int l) { return s > t && l == m; });
    return k >= 0 ? b.eadj[(size_t)v * b.cap + k] : 0.0;
}

__device__ __forceinline__ int entry_at(const BwdDev &b, int v, int t) {
    return route_find(b, v, 0, [&](int s, int) { return s == t; });
}

// copy the state at the start of step (t0 + rec) into the tape
__global__ void k_tape_pre(DevSim d, BwdDev b, int rec, int cur) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float *pc = cur ? d.pos1 : d.pos0;
    if (i < b.S) {
        b.tpos[(size_t)rec * b.S + i] = pc[i];
        b.tvid[(size_t)rec * b.S + i] = d.saux[i].x;
    }
    if (i < d.L) b.tlq[(size_t)rec * d.L + i] = d.lq[i];
}

// adjoint of the final positions (vehicles on a link at the end of the rollout)
__global__ void k_bwd_init(DevSim d, BwdDev b, const float *dxT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    b.xbar[i] = (dxT && d.vstate[i] >= 0) ? (double)dxT[i] : 0.0;
}

// (1) observation at time t + 1 = the state of tape record rec: one warp per link
__global__ void k_bwd_obs(DevSim d, BwdDev b, int rec, int bin) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= d.L) return;
    const double cb = b.Cbar[(size_t)bin * d.L + j];
    if (cb == 0.0) return;
    const int4 q = b.tlq[(size_t)rec * d.L + j];
    const int4 st = d.lst[j];
    const double len = (double)d.geo[j].x, s5 = 5.0 / len, half = 0.5 * len;
    for (int k = lane; k < q.y; k += 32) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        const size_t o = (size_t)rec * b.S + st.x + idx;
        const int v = b.tvid[o];
        const double x = (double)b.tpos[o];
        const double sg = 1.0 / (1.0 + exp(-s5 * (x - half)));
        b.xbar[v] += cb * s5 * sg * (1.0 - sg);
        if (x >= half) {
            const int k2 = b.od[v];
            atomicAdd(&b.glam[k2], cb / (double)b.od_lambda[k2]);
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

// (2a) merge candidates of step t: abar, softmax weight, per-target sums
__global__ void k_bwd_node_z(DevSim d, BwdDev b, int t, int rec, int bin0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.L + d.V) return;
    const Cand c = load_cand(d, b, i, rec);
    if (c.vid < 0) return;
    const int v = c.vid;
    if (i < d.L && (c.won || c.tgt == kTgtSink)) {          // an exit from link i
        const int k2 = b.od[v];
        atomicAdd(&b.glam[k2], b.Csuf[(size_t)bin0 * d.L + i] / (double)b.od_lambda[k2]);
    }
    int rw = -1;
    if (c.won) {                                             // adjoint right after this entry
        rw = entry_at(b, v, t);
        if (rw >= 0) b.eadj[(size_t)v * b.cap + rw] = b.xbar[v];
    }
    if (c.tgt < 0) return;
    const double key = ((double)c.alpha + (double)gumbel(d.key0, d.key1, v, t, 1, 0)) * (double)b.inv_tau;
    const double kmax = (double)merge_key_of(b.tW[(size_t)rec * d.L + c.tgt]) * (double)b.inv_tau;
    const double e = exp(key - kmax);
    double Enew, Xold;
    if (c.won) {
        Enew = b.xbar[v];
        Xold = 0.0;
        if (i < d.L && rw >= 0) {                            // next re-entry into the source link
            const int k = route_find(b, v, rw + 1, [&](int, int l) { return l == i; });
            if (k >= 0) Xold = b.eadj[(size_t)v * b.cap + k];
        }
    } else {
        Enew = next_entry(b, v, c.tgt, t);
        Xold = b.xbar[v];
    }
    const double abar = (double)d.M * (Enew - Xold) - (double)c.x * Xold;
    const size_t eo = (size_t)(t & 1) * (d.L + d.V) + i;
    b.ebuf[eo] = e;
    b.abuf[eo] = abar;
    const size_t zo = (size_t)(t & 1) * d.L + c.tgt;
    atomicAdd(&b.Z[zo], e);
    atomicAdd(&b.SA[zo], e * abar);
}

// (2b) merge and link-choice Jacobians of step t
__global__ void k_bwd_node_g(DevSim d, BwdDev b, int t, int rec) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.L + d.V) return;
    const Cand c = load_cand(d, b, i, rec);
    if (c.vid < 0 || c.tgt < 0) return;
    const size_t zo = (size_t)(t & 1) * d.L + c.tgt;
    const double Z = b.Z[zo];
    const size_t eo = (size_t)(t & 1) * (d.L + d.V) + i;
    const double pi = b.ebuf[eo] / Z;
    const double S = b.SA[zo] / Z;
    const double vbar = pi * (b.abuf[eo] - S) * (double)b.inv_tau;   // adjoint of V'_i
    if (i < d.L) atomicAdd(&b.ga[i], vbar); else atomicAdd(b.gao, vbar);
    const double lbar = (double)c.alpha * vbar;                      // adjoint of l_i at the target
    if (lbar == 0.0) return;
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
    // keys (V_k + g_k)/tau of the first kG slots held in registers (fully
    // unrolled); slots past kG are recomputed where needed
    constexpr int kG = 8;
    auto keyk = [&](int k, int &m, float &df) {
        const float4 e = info[k];
        m = __float_as_int(e.w);
        df = d.dest_feat[(size_t)zone * d.V + __float_as_int(e.z)];
        const float util = __fadd_rn(e.x, __fmul_rn(e.y, df));
        return ((double)util + (double)gumbel(d.key0, d.key1, v, t, 0, k)) * (double)b.inv_tau;
    };
    double key[kG];
    float dfs[kG];
    int ms[kG];
    double kmax = -INFINITY;
    int ks = 0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            key[k] = keyk(k, ms[k], dfs[k]);
            kmax = fmax(kmax, key[k]);
            if (ms[k] == c.tgt) ks = k;
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const double kk = keyk(k, m, df);
        kmax = fmax(kmax, kk);
        if (m == c.tgt) ks = k;
    }
    double zs = 0.0, eks = 0.0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            key[k] = exp(key[k] - kmax);
            zs += key[k];
            if (k == ks) eks = key[k];
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const double ek = exp(keyk(k, m, df) - kmax);
        zs += ek;
        if (k == ks) eks = ek;
    }
    const double pks = eks / zs;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        if (k < deg) {
            const double pk = key[k] / zs;
            const double Vbar = pk * ((k == ks ? 1.0 : 0.0) - pks) * lbar * (double)b.inv_tau;
            atomicAdd(&b.gU[ms[k]], Vbar);
            atomicAdd(&b.gG[ms[k]], Vbar * (double)dfs[k]);
        }
    }
    for (int k = kG; k < deg; ++k) {
        int m;
        float df;
        const double pk = exp(keyk(k, m, df) - kmax) / zs;
        const double Vbar = pk * ((k == ks ? 1.0 : 0.0) - pks) * lbar * (double)b.inv_tau;
        atomicAdd(&b.gU[m], Vbar);
        atomicAdd(&b.gG[m], Vbar * (double)df);
    }
}

// (3) car-following of step (t0 + rec): one warp per link; an iteration covers
// kCfR rounds of 32 queue positions (leader first), issuing every tape and
// adjoint load of them (and of the vehicle after them) before using any.
// Vehicle k's adjoint at time t is its own adjoint at t + 1 unless its update
// was congested (then x' depended on the leader only), plus its follower's
// adjoint when the follower was congested (the follower's headway used x_k).
// The follower's values come from the next lane, or for lane 31 from lane 0 of
// the next round.  Every adjoint an iteration reads is read before any lane
// writes, and a link's vehicles belong to its warp only.  Per-link parameter
// sums: free -> u (x' = x + u dt), congested -> s.
constexpr int kBwdCfThreads = 256;
constexpr int kCfR = 2;

__global__ void __launch_bounds__(kBwdCfThreads) k_bwd_cf(DevSim d, BwdDev b, int rec, int t) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * kBwdCfThreads + threadIdx.x) >> 5;
    if (j >= d.L) return;
    if (lane == 0) {                                        // merge sums of step t - 1 start from zero
        const size_t zo = (size_t)((t + 1) & 1) * d.L + j;
        b.Z[zo] = 0.0;
        b.SA[zo] = 0.0;
    }
    const int4 q = b.tlq[(size_t)rec * d.L + j];
    const int4 st = d.lst[j];                               // issued with the queue state
    const int n = q.y;
    if (n == 0) return;
    const double dt = (double)d.dt;
    const size_t tb = (size_t)rec * b.S + st.x;
    auto slot = [&](int k) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        return idx;
    };
    double su = 0.0, ss = 0.0;
    for (int k0 = 0; k0 < n; k0 += 32 * kCfR) {
        int v[kCfR], tag[kCfR];
        double g[kCfR];
#pragma unroll
        for (int r = 0; r < kCfR; ++r) {
            const int k = k0 + 32 * r + lane;
            v[r] = -1;
            tag[r] = kTagStop;
            if (k < n) {
                const int idx = slot(k);
                v[r] = b.tvid[tb + idx];
                tag[r] = b.ttag[tb + idx];
            }
        }
        const int kx = k0 + 32 * kCfR;                      // the vehicle after this iteration
        int vx = -1, tx = kTagStop;
        if (lane == 0 && kx < n) {
            const int idx = slot(kx);
            vx = b.tvid[tb + idx];
            tx = b.ttag[tb + idx];
        }
#pragma unroll
        for (int r = 0; r < kCfR; ++r) g[r] = v[r] >= 0 ? b.xbar[v[r]] : 0.0;
        const double gx = vx >= 0 ? b.xbar[vx] : 0.0;
        double pre[kCfR];
#pragma unroll
        for (int r = 0; r < kCfR; ++r) {
            int ftag = __shfl_down_sync(kFull, tag[r], 1);
            double fg = __shfl_down_sync(kFull, g[r], 1);
            const int ntag = __shfl_sync(kFull, r + 1 < kCfR ? tag[r + 1 < kCfR ? r + 1 : r] : tx, 0);
            const double ng = __shfl_sync(kFull, r + 1 < kCfR ? g[r + 1 < kCfR ? r + 1 : r] : gx, 0);
            if (lane == 31) {
                ftag = ntag;
                fg = ng;
            }
            const int k = k0 + 32 * r + lane;
            pre[r] = 0.0;
            if (k < n) {
                pre[r] = (tag[r] == kTagCong) ? 0.0 : g[r];
                if (k + 1 < n && ftag == kTagCong) pre[r] += fg;
                if (tag[r] == kTagFree) su += g[r] * dt;
                if (tag[r] == kTagCong) ss -= g[r];
            }
        }
        __syncwarp();                                       // every lane has read before any writes
#pragma unroll
        for (int r = 0; r < kCfR; ++r)
            if (v[r] >= 0) b.xbar[v[r]] = pre[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(kFull, su, o);
        ss += __shfl_xor_sync(kFull, ss, o);
    }
    if (lane == 0) {
        if (su != 0.0) b.gu[j] += su;
        if (ss != 0.0) b.gs[j] += ss;
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
