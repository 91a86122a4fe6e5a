// trafficsim.cu -- forward step kernels and the C ABI of include/trafficsim.h.
//
// One step phi = g o f runs as two kernels:
//   step_fwd_a  one warp per link: observation (when a bin closes), Newell
//               car-following of the whole queue (SI-A, Eq. newell_model) from
//               the time-t positions into the other position buffer, outflow
//               credit, leader arrival test (Alg. S2), link choice over the
//               choice set by Gumbel argmax with one lane per candidate link
//               (SI-B Eqs. softmax/gumbel/straigththrough), and the merge
//               (SI-B "Merge choice") as a 64-bit atomicMax of (alpha + g',
//               ~vehicle id) into the target's word.  One lane per origin node
//               does the same for the head of its origin queue.
//   step_fwd_b  one thread per link / origin node: applies the transfers of the
//               step (SI-B Eq. transfer): pops the leader that won or left to
//               its destination, pushes the winner at x = 0, updates credit,
//               exits and link times, and precomputes the vacancy flag
//               X_min > dn/kappa for the next step from the post-f position of
//               the new queue tail.
// A rollout is captured once per horizon into a CUDA graph of 2T + 1 kernels.
#include "ts_sim.cuh"
#include "../../include/trafficsim.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

using namespace ts;

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------

// Derived per-link quantities from the differentiable parameters.
__global__ void k_params(DevSim d, const float *len, const float *u, const float *kappa,
                         const float *beta, const float *cost, const float *phi,
                         const float *psi, const float *w, const int *head, float dn,
                         float eps_tag) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.L) return;
    const float L = len[j];
    const float s = __fdiv_rn(dn, kappa[j]);
    const float udt = __fmul_rn(u[j], d.dt);
    const float dtag = __fmul_rn(eps_tag, __fadd_rn(1.0f, L));
    float a = __fdiv_rn(beta[j], cost[j]);
    float g = 0.0f;
    for (int f = 0; f < d.F; ++f) {
        const float wf = w[f];
        a = __fadd_rn(a, __fmul_rn(wf, phi[(size_t)j * d.F + f]));
        g = __fadd_rn(g, __fmul_rn(wf, psi[(size_t)j * d.F + f]));
    }
    const_cast<float4 *>(d.geo)[j] = make_float4(L, udt, s, dtag);
    const_cast<float4 *>(d.tinfo)[j] = make_float4(a, g, __int_as_float(head[j]), __fmul_rn(L, 0.5f));
}

__global__ void k_reset(DevSim d, const int *fifo_beg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.L) {
        const int4 st = d.lst[i];
        d.lq[i] = make_int4(0, 0, st.w, 0);
        d.vac[i] = 1;
        d.W0[i] = 0ull;
        d.W1[i] = 0ull;
        d.acc_dx[i] = 0.0f; d.acc_n[i] = 0; d.tt_sum[i] = 0; d.tt_cnt[i] = 0; d.C_prev[i] = 0;
        d.cand_tgt[i] = kTgtNone; d.cand_vid[i] = -1;
    }
    if (i < d.V) { d.fifo_ptr[i] = fifo_beg[i]; d.ncand_tgt[i] = kTgtNone; d.ncand_vid[i] = -1; }
    if (i < d.N) { d.vstate[i] = kVehWaiting; d.entry[i] = 0; }
    if (i < 4) d.err[i] = 0;
}

// Returns (on lane 0) 1 if the link's leader was a candidate of the node model.
__device__ __forceinline__ int link_warp(const DevSim &d, int j, int lane, int t, bool obs_only) {
    const int p = t & 1;
    const float *pc = p ? d.pos1 : d.pos0;
    float *pn = p ? d.pos0 : d.pos1;
    const int4 q = d.lq[j];
    const int4 st = d.lst[j];
    if (obs_only || (t > 0 && t % d.obs_every == 0)) {
        observe_link(d, j, lane, t, q, st, pc);
        if (obs_only) return 0;
    }
    const float4 g = d.geo[j];
    const int n = q.y;
    // ---- f: car-following of the queue, leader first ----
    float xl = 0.0f, accdx = 0.0f, carry = 0.0f;
    for (int base = 0; base < n; base += 32) {
        const int k = base + lane;
        float x = 0.0f;
        int slot = 0;
        if (k < n) {
            int idx = q.x + k;
            if (idx >= st.y) idx -= st.y;
            slot = st.x + idx;
            x = pc[slot];
        }
        float xa = __shfl_up_sync(kFull, x, 1);
        if (lane == 0) xa = carry;
        if (k < n) {
            const float h = (k == 0) ? d.M : __fsub_rn(xa, x);
            int tag;
            const float xn = newell(x, h, g.x, g.y, g.z, g.w, tag);
            pn[slot] = xn;
            if (d.tag_tape) d.tag_tape[slot] = (int8_t)tag;
            accdx += __fsub_rn(xn, x);
            if (k == 0) xl = xn;
        }
        carry = __shfl_sync(kFull, x, 31);
    }
    accdx = warp_sumf(accdx);
    // ---- g: credit, arrival, choice, merge ----
    int cand = 0, vid = -1, z = 0, credit = 0;
    int4 nd = make_int4(0, 0, 0, 0);
    if (lane == 0) {
        if (n > 0) { d.acc_dx[j] += accdx; d.acc_n[j] += n; }
        credit = min(q.z + st.z, st.w);
        reinterpret_cast<int *>(&d.lq[j])[2] = credit;
        cand = (n > 0) && (xl >= __fsub_rn(g.x, d.eps_arr)) && (credit >= d.dn_fx);
        if (cand) {
            vid = d.svid[st.x + q.x];
            z = d.dest_zone[vid];
            nd = d.lnode[j];
        }
        d.cand_vid[j] = cand ? vid : -1;
        if (!cand) d.cand_tgt[j] = kTgtNone;
        else if (nd.y == z) { d.cand_tgt[j] = kTgtSink; cand = 0; }
    }
    const int counted = (lane == 0) ? (d.cand_vid[j] >= 0) : 0;
    cand = __shfl_sync(kFull, cand, 0);
    if (!cand) return counted;
    vid = __shfl_sync(kFull, vid, 0);
    z = __shfl_sync(kFull, z, 0);
    nd.z = __shfl_sync(kFull, nd.z, 0);
    nd.w = __shfl_sync(kFull, nd.w, 0);
    const int deg = nd.w - nd.z;
    float key = -INFINITY;
    int m = -1;
    if (lane < deg) {
        m = d.lo_idx[nd.z + lane];
        key = choice_key(d, m, z, vid, t, lane);
    }
    // argmax over lanes, ties to the lowest slot
    int best = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ok = __shfl_xor_sync(kFull, key, o);
        const int ob = __shfl_xor_sync(kFull, best, o);
        if (ok > key || (ok == key && ob < best)) { key = ok; best = ob; }
    }
    const int mt = __shfl_sync(kFull, m, best);
    if (lane == 0) {
        if (d.vac[mt]) {
            const float kp = __fadd_rn(d.alpha[j], gumbel(d.key0, d.key1, vid, t, 1, 0));
            atomicMax(p ? &d.W1[mt] : &d.W0[mt], merge_word(kp, vid));
            d.cand_tgt[j] = mt;
        } else {
            d.cand_tgt[j] = kTgtBlocked;
        }
    }
    return counted;
}

// Head of the origin queue of node n (a virtual inflow link of length 0).
// Returns 1 if the node's origin queue had a candidate.
__device__ __forceinline__ int node_lane(const DevSim &d, int n, int t) {
    const int p = t & 1;
    const int ptr = d.fifo_ptr[n];
    int tgt = kTgtNone, cv = -1;
    if (ptr < d.fifo_end[n] && d.fifo_dep[ptr] <= t) {
        cv = d.fifo_list[ptr];
        const int z = d.dest_zone[cv];
        if (d.node_zone[n] == z) {
            tgt = kTgtSink;
        } else {
            const int b = d.no_ptr[n], e = d.no_ptr[n + 1];
            float bk = 0.0f;
            int mt = -1;
            for (int k = 0; k < e - b; ++k) {
                const int m = d.no_idx[b + k];
                const float key = choice_key(d, m, z, cv, t, k);
                if (mt < 0 || key > bk) { bk = key; mt = m; }
            }
            if (d.vac[mt]) {
                const float kp = __fadd_rn(d.alpha[d.L], gumbel(d.key0, d.key1, cv, t, 1, 0));
                atomicMax(p ? &d.W1[mt] : &d.W0[mt], merge_word(kp, cv));
                tgt = mt;
            } else {
                tgt = kTgtBlocked;
            }
        }
    }
    d.ncand_vid[n] = cv;
    d.ncand_tgt[n] = tgt;
    return cv >= 0;
}

__global__ void __launch_bounds__(128) k_step_a(DevSim d, int t, int obs_only) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    int nc = 0;
    if (gw < d.L) {
        nc = link_warp(d, gw, lane, t, obs_only != 0);
    } else if (!obs_only) {
        const int n = (gw - d.L) * 32 + lane;
        if (n < d.V) nc = node_lane(d, n, t);
        nc = warp_sum(nc);
    }
    if (lane == 0 && nc) atomicAdd(&d.step_delta[4 * t + 2], nc);
}

__global__ void __launch_bounds__(256) k_step_b(DevSim d, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = t & 1;
    const unsigned long long *W = p ? d.W1 : d.W0;
    int released = 0, arrived = 0, entered = 0;
    if (i < d.L) {
        const int j = i;
        float *pn = p ? d.pos0 : d.pos1;
        int4 q = d.lq[j];
        const int4 st = d.lst[j];
        const int tgt = d.cand_tgt[j];
        const int cv = d.cand_vid[j];
        bool out = false;
        if (tgt == kTgtSink) {
            out = true;
            d.vstate[cv] = kVehArrived;
            arrived = 1;
        } else if (tgt >= 0) {
            const unsigned long long w = W[tgt];
            out = (w != 0ull) && merge_vid(w) == cv;
        }
        if (out) {
            d.tt_sum[j] += t + 1 - d.entry[cv];
            d.tt_cnt[j] += 1;
            q.x = (q.x + 1 == st.y) ? 0 : q.x + 1;
            q.y -= 1;
            q.z -= d.dn_fx;
            q.w += 1;
        }
        const unsigned long long win = W[j];
        if (win != 0ull) {
            const int v = merge_vid(win);
            if (q.y >= st.y) {
                set_error(d, SIM_EOVERFLOW, j, t);
            } else {
                int idx = q.x + q.y;
                if (idx >= st.y) idx -= st.y;
                pn[st.x + idx] = 0.0f;
                d.svid[st.x + idx] = v;
                q.y += 1;
                d.entry[v] = t + 1;
                d.vstate[v] = j;
                entered = 1;
            }
        }
        (p ? d.W0 : d.W1)[j] = 0ull;
        d.lq[j] = q;
        // vacancy of the coming step: post-f position of the queue tail > s
        int vac = 1;
        if (q.y > 0) {
            const float4 g = d.geo[j];
            int it = q.x + q.y - 1;
            if (it >= st.y) it -= st.y;
            const float xt = pn[st.x + it];
            float h = d.M;
            if (q.y > 1) {
                int ip = it - 1;
                if (ip < 0) ip += st.y;
                h = __fsub_rn(pn[st.x + ip], xt);
            }
            int tag;
            vac = newell(xt, h, g.x, g.y, g.z, g.w, tag) > g.z;
        }
        d.vac[j] = vac;
    } else if (i < d.L + d.V) {
        const int n = i - d.L;
        const int tgt = d.ncand_tgt[n];
        const int cv = d.ncand_vid[n];
        if (tgt == kTgtSink) {
            d.fifo_ptr[n] += 1;
            d.vstate[cv] = kVehArrived;
            released = 1;
            arrived = 1;
        } else if (tgt >= 0) {
            const unsigned long long w = W[tgt];
            if (w != 0ull && merge_vid(w) == cv) { d.fifo_ptr[n] += 1; released = 1; }
        }
    }
    released = warp_sum(released);
    arrived = warp_sum(arrived);
    entered = warp_sum(entered);
    if ((threadIdx.x & 31) == 0) {
        if (released) atomicAdd(&d.step_delta[4 * t], released);
        if (arrived) atomicAdd(&d.step_delta[4 * t + 1], arrived);
        if (entered) atomicAdd(&d.step_delta[4 * t + 3], entered);
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------

struct sim_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevSim d{};
    // sizes
    int V = 0, L = 0, N = 0, F = 0, Z = 0, n_od = 0, S = 0;
    sim_options opt{};
    // host copies
    std::vector<int> tail, head, lst_host, fifo_beg, fifo_list;
    std::vector<float> length, u, kappa, alpha, beta, cost, w, phi, psi;
    float alpha_origin = 2.505f;
    // raw device inputs for k_params
    float *d_len = nullptr, *d_u = nullptr, *d_kappa = nullptr, *d_beta = nullptr, *d_cost = nullptr;
    float *d_phi = nullptr, *d_psi = nullptr, *d_w = nullptr;
    int *d_head = nullptr, *d_fifo_beg = nullptr;
    std::vector<void *> allocs;
    size_t bytes = 0;
    // run state
    int t = 0, T = 0, n_bins = 0;
    bool reset_done = false;
    int cap_T = 0;                       // capacity of the per-T output buffers
    std::map<int, cudaGraphExec_t> graphs;
    std::string err;
};

static std::string g_create_err;

static int fail(sim_ctx *h, int code, const std::string &msg) {
    if (h) h->err = msg; else g_create_err = msg;
    return code;
}

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return fail(h, SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static int dalloc(sim_ctx *h, T **p, size_t n) {
    void *q = nullptr;
    size_t b = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, b);
    if (e != cudaSuccess) return fail(h, SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->allocs.push_back(q);
    h->bytes += b;
    *p = (T *)q;
    return SIM_OK;
}

template <class T>
static int upload(sim_ctx *h, T **p, const T *src, size_t n) {
    int rc = dalloc(h, p, n);
    if (rc) return rc;
    if (n) CU(cudaMemcpyAsync(*p, src, n * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return SIM_OK;
}

#define TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

extern "C" int32_t sim_n_bins(int32_t T, int32_t obs_every) {
    if (T <= 0 || obs_every <= 0) return 0;
    return (T + obs_every - 1) / obs_every;
}

static int upload_params(sim_ctx *h, const sim_params *par) {
    const int L = h->L, F = h->F;
    for (int j = 0; j < L; ++j) {
        if (!(par->u[j] > 0.0f) || !std::isfinite(par->u[j])) return fail(h, SIM_EINVAL, "u must be positive");
        if (!(par->kappa[j] > 0.0f) || !std::isfinite(par->kappa[j])) return fail(h, SIM_EINVAL, "kappa must be positive");
        if (!(par->cost[j] > 0.0f) || !std::isfinite(par->cost[j])) return fail(h, SIM_EINVAL, "cost must be positive");
        if (!std::isfinite(par->alpha[j]) || !std::isfinite(par->beta[j])) return fail(h, SIM_EINVAL, "alpha/beta must be finite");
    }
    for (int f = 0; f < F; ++f)
        if (!std::isfinite(par->w[f])) return fail(h, SIM_EINVAL, "w must be finite");
    h->u.assign(par->u, par->u + L);
    h->kappa.assign(par->kappa, par->kappa + L);
    h->alpha.assign(par->alpha, par->alpha + L);
    h->beta.assign(par->beta, par->beta + L);
    h->cost.assign(par->cost, par->cost + L);
    h->w.assign(par->w, par->w + F);
    h->alpha_origin = par->alpha_origin;
    CU(cudaMemcpyAsync(h->d_u, par->u, L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->d_kappa, par->kappa, L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(const_cast<float *>(h->d.alpha), par->alpha, L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(const_cast<float *>(h->d.alpha) + L, &h->alpha_origin, sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->d_beta, par->beta, L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->d_cost, par->cost, L * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    if (F) CU(cudaMemcpyAsync(h->d_w, par->w, F * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    k_params<<<(L + 255) / 256, 256, 0, h->stream>>>(h->d, h->d_len, h->d_u, h->d_kappa, h->d_beta, h->d_cost,
                                                     h->d_phi, h->d_psi, h->d_w, h->d_head, h->opt.dn,
                                                     h->opt.eps_tag);
    CU(cudaGetLastError());
    // the captured graphs read the parameters from device memory and stay valid;
    // host copies of the parameters must outlive the asynchronous uploads
    CU(cudaStreamSynchronize(h->stream));
    h->reset_done = false;
    return SIM_OK;
}

static int create_impl(sim_ctx *h, const sim_network *net, const sim_demand *dem, const sim_params *par,
                       const sim_options *opt) {
    if (!net || !dem || !par || !opt) return fail(h, SIM_EINVAL, "null argument");
    const int V = net->V, L = net->L, N = dem->N, F = net->F, Z = net->Z;
    if (V <= 0 || L <= 0 || N < 0 || F < 0 || Z <= 0) return fail(h, SIM_EINVAL, "bad sizes");
    if (!(opt->dt > 0) || !(opt->dn > 0) || opt->obs_every <= 0 || !(opt->tau_gumbel > 0))
        return fail(h, SIM_EINVAL, "bad options");
    h->V = V; h->L = L; h->N = N; h->F = F; h->Z = Z; h->n_od = dem->n_od;
    h->opt = *opt;
    h->device = opt->device;
    for (int j = 0; j < L; ++j) {
        if (net->tail[j] < 0 || net->tail[j] >= V || net->head[j] < 0 || net->head[j] >= V)
            return fail(h, SIM_EINVAL, "link endpoint out of range");
        if (!(net->length[j] > 0.0f) || !std::isfinite(net->length[j])) return fail(h, SIM_EINVAL, "length must be positive");
        if (net->q_fx[j] <= 0) return fail(h, SIM_EINVAL, "capacity must be positive");
    }
    for (int n = 0; n < V; ++n)
        if (net->node_zone[n] < 0 || net->node_zone[n] >= Z) return fail(h, SIM_EINVAL, "node zone out of range");
    for (size_t k = 0; k < (size_t)Z * V; ++k)
        if (!std::isfinite(net->dest_feat[k])) return fail(h, SIM_EINVAL, "destination feature not finite");
    for (size_t k = 0; k < (size_t)L * F; ++k)
        if (!std::isfinite(net->phi[k]) || !std::isfinite(net->psi[k])) return fail(h, SIM_EINVAL, "feature not finite");
    for (int i = 0; i < N; ++i) {
        if (dem->origin[i] < 0 || dem->origin[i] >= V) return fail(h, SIM_EINVAL, "origin out of range");
        if (dem->dest_zone[i] < 0 || dem->dest_zone[i] >= Z) return fail(h, SIM_EINVAL, "destination zone out of range");
        if (dem->dep_step[i] < 0) return fail(h, SIM_EINVAL, "negative departure step");
    }
    h->tail.assign(net->tail, net->tail + L);
    h->head.assign(net->head, net->head + L);
    h->length.assign(net->length, net->length + L);
    // out-links of each node in increasing link id
    std::vector<int> no_ptr(V + 1, 0), no_idx(L);
    for (int j = 0; j < L; ++j) no_ptr[net->tail[j] + 1]++;
    for (int n = 0; n < V; ++n) no_ptr[n + 1] += no_ptr[n];
    {
        std::vector<int> fill(V, 0);
        for (int j = 0; j < L; ++j) no_idx[no_ptr[net->tail[j]] + fill[net->tail[j]]++] = j;
    }
    for (int n = 0; n < V; ++n) {
        if (no_ptr[n + 1] == no_ptr[n]) return fail(h, SIM_EINVAL, "node without out-link (dead end)");
        if (no_ptr[n + 1] - no_ptr[n] > 32) return fail(h, SIM_EINVAL, "node out-degree above 32");
    }
    // choice set after each link: U-turns removed unless they are the only way out
    std::vector<int> lnode(4 * L), lo_idx;
    lo_idx.reserve(L * 3);
    for (int l = 0; l < L; ++l) {
        const int n = net->head[l];
        int c = 0;
        for (int k = no_ptr[n]; k < no_ptr[n + 1]; ++k) c += net->head[no_idx[k]] != net->tail[l];
        lnode[4 * l + 0] = n;
        lnode[4 * l + 1] = net->node_zone[n];
        lnode[4 * l + 2] = (int)lo_idx.size();
        for (int k = no_ptr[n]; k < no_ptr[n + 1]; ++k) {
            const int m = no_idx[k];
            if (!c || net->head[m] != net->tail[l]) lo_idx.push_back(m);
        }
        lnode[4 * l + 3] = (int)lo_idx.size();
    }
    // queue arenas: capacity floor(L kappa / dn) + 2 slots per link
    std::vector<int> lst(4 * L);
    long long S = 0;
    const long long dn_fx = llrint((double)opt->dn * SIM_FX_ONE);
    for (int j = 0; j < L; ++j) {
        const double cap = std::floor((double)net->length[j] * (double)par->kappa[j] / (double)opt->dn) + 2.0;
        lst[4 * j + 0] = (int)S;
        lst[4 * j + 1] = (int)cap;
        lst[4 * j + 2] = net->q_fx[j];
        lst[4 * j + 3] = (int)std::max<long long>(net->q_fx[j], dn_fx);
        S += (long long)cap;
    }
    if (S > (1ll << 30)) return fail(h, SIM_EINVAL, "queue arena too large");
    h->S = (int)S;
    h->lst_host = lst;
    // origin queues sorted by (origin, departure step, id)
    std::vector<int> fifo(N), fifo_beg(V + 1, 0), fifo_dep(N);
    std::iota(fifo.begin(), fifo.end(), 0);
    std::stable_sort(fifo.begin(), fifo.end(), [&](int a, int b) {
        if (dem->origin[a] != dem->origin[b]) return dem->origin[a] < dem->origin[b];
        if (dem->dep_step[a] != dem->dep_step[b]) return dem->dep_step[a] < dem->dep_step[b];
        return a < b;
    });
    for (int i = 0; i < N; ++i) fifo_beg[dem->origin[i] + 1]++;
    for (int n = 0; n < V; ++n) fifo_beg[n + 1] += fifo_beg[n];
    for (int k = 0; k < N; ++k) fifo_dep[k] = dem->dep_step[fifo[k]];
    std::vector<int> fifo_end(fifo_beg.begin() + 1, fifo_beg.end());
    h->fifo_beg = fifo_beg;
    h->fifo_list = fifo;

    CU(cudaSetDevice(h->device));
    if (opt->stream) {
        h->stream = (cudaStream_t)opt->stream;
    } else {
        CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    DevSim &d = h->d;
    d.V = V; d.L = L; d.N = N; d.Z = Z; d.F = F;
    d.dn_fx = (int)dn_fx;
    d.obs_every = opt->obs_every;
    d.M = opt->M; d.eps_arr = opt->eps_arr; d.dt = opt->dt;
    d.key0 = (uint32_t)(opt->seed & 0xffffffffull);
    d.key1 = (uint32_t)(opt->seed >> 32) ^ opt->scenario_id;
    float4 *geo, *tinfo;
    int4 *lstd, *lnoded;
    TRY(dalloc(h, &geo, L)); d.geo = geo;
    TRY(dalloc(h, &tinfo, L)); d.tinfo = tinfo;
    TRY(upload(h, &lstd, (const int4 *)lst.data(), L)); d.lst = lstd;
    TRY(upload(h, &lnoded, (const int4 *)lnode.data(), L)); d.lnode = lnoded;
    float *alpha_d;
    TRY(dalloc(h, &alpha_d, L + 1)); d.alpha = alpha_d;     // [L] = origin queues
    int *p;
    TRY(upload(h, &p, lo_idx.data(), lo_idx.size())); d.lo_idx = p;
    TRY(upload(h, &p, no_ptr.data(), no_ptr.size())); d.no_ptr = p;
    TRY(upload(h, &p, no_idx.data(), no_idx.size())); d.no_idx = p;
    TRY(upload(h, &p, net->node_zone, V)); d.node_zone = p;
    TRY(upload(h, &p, fifo_end.data(), V)); d.fifo_end = p;
    TRY(upload(h, &p, fifo.data(), N)); d.fifo_list = p;
    TRY(upload(h, &p, fifo_dep.data(), N)); d.fifo_dep = p;
    TRY(upload(h, &p, dem->dest_zone, N)); d.dest_zone = p;
    float *fp;
    TRY(upload(h, &fp, net->dest_feat, (size_t)Z * V)); d.dest_feat = fp;
    TRY(upload(h, &h->d_fifo_beg, fifo_beg.data(), V));
    TRY(upload(h, &h->d_len, net->length, L));
    TRY(upload(h, &h->d_head, net->head, L));
    TRY(upload(h, &h->d_phi, net->phi, (size_t)L * F));
    TRY(upload(h, &h->d_psi, net->psi, (size_t)L * F));
    h->phi.assign(net->phi, net->phi + (size_t)L * F);
    h->psi.assign(net->psi, net->psi + (size_t)L * F);
    TRY(dalloc(h, &h->d_u, L));
    TRY(dalloc(h, &h->d_kappa, L));
    TRY(dalloc(h, &h->d_beta, L));
    TRY(dalloc(h, &h->d_cost, L));
    TRY(dalloc(h, &h->d_w, std::max(F, 1)));
    // dynamic state
    TRY(dalloc(h, &d.lq, L));
    TRY(dalloc(h, &d.vac, L));
    TRY(dalloc(h, &d.pos0, S));
    TRY(dalloc(h, &d.pos1, S));
    TRY(dalloc(h, &d.svid, S));
    TRY(dalloc(h, &d.W0, L));
    TRY(dalloc(h, &d.W1, L));
    TRY(dalloc(h, &d.cand_vid, L));
    TRY(dalloc(h, &d.cand_tgt, L));
    TRY(dalloc(h, &d.ncand_vid, V));
    TRY(dalloc(h, &d.ncand_tgt, V));
    TRY(dalloc(h, &d.fifo_ptr, V));
    TRY(dalloc(h, &d.entry, N));
    TRY(dalloc(h, &d.vstate, N));
    TRY(dalloc(h, &d.acc_dx, L));
    TRY(dalloc(h, &d.acc_n, L));
    TRY(dalloc(h, &d.tt_sum, L));
    TRY(dalloc(h, &d.tt_cnt, L));
    TRY(dalloc(h, &d.C_prev, L));
    TRY(dalloc(h, &d.err, 4));
    CU(cudaMemsetAsync(d.pos0, 0, (size_t)S * sizeof(float), h->stream));
    CU(cudaMemsetAsync(d.pos1, 0, (size_t)S * sizeof(float), h->stream));
    CU(cudaMemsetAsync(d.svid, 0xff, (size_t)S * sizeof(int), h->stream));
    d.tag_tape = nullptr;
    TRY(upload_params(h, par));
    CU(cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

static void release(sim_ctx *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    h->graphs.clear();
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
}

extern "C" int sim_create(const sim_network *net, const sim_demand *dem, const sim_params *par,
                          const sim_options *opt, sim_handle *out) {
    if (!out) return fail(nullptr, SIM_EINVAL, "null output handle");
    *out = nullptr;
    sim_ctx *h = new sim_ctx();
    int rc = create_impl(h, net, dem, par, opt);
    if (rc) {
        g_create_err = h->err;
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return SIM_OK;
}

extern "C" int sim_set_params(sim_handle h, const sim_params *par) {
    if (!h || !par) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    return upload_params(h, par);
}

// per-horizon buffers: outputs and step counters
static int ensure_T(sim_ctx *h, int T) {
    if (T <= h->cap_T) return SIM_OK;
    // outputs are re-pointed: cached graphs bake the old pointers
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    h->graphs.clear();
    const int nb = sim_n_bins(T, h->opt.obs_every);
    TRY(dalloc(h, &h->d.out_counts, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.out_speed, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.out_tt, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.step_delta, (size_t)4 * T));
    h->cap_T = T;
    return SIM_OK;
}

static void enqueue_reset(sim_ctx *h, int T) {
    const int nmax = std::max(std::max(h->L, h->V), std::max(h->N, 4));
    cudaMemsetAsync(h->d.step_delta, 0, (size_t)4 * T * sizeof(int), h->stream);
    const int nb = sim_n_bins(T, h->opt.obs_every);
    cudaMemsetAsync(h->d.out_counts, 0, (size_t)nb * h->L * sizeof(int), h->stream);
    k_reset<<<(nmax + 255) / 256, 256, 0, h->stream>>>(h->d, h->d_fifo_beg);
}

static void enqueue_step(sim_ctx *h, int t) {
    const int warps = h->L + (h->V + 31) / 32;
    k_step_a<<<(warps * 32 + 127) / 128, 128, 0, h->stream>>>(h->d, t, 0);
    k_step_b<<<(h->L + h->V + 255) / 256, 256, 0, h->stream>>>(h->d, t);
}

static void enqueue_obs_final(sim_ctx *h, int T) {
    k_step_a<<<(h->L * 32 + 127) / 128, 128, 0, h->stream>>>(h->d, T, 1);
}

static int check_device_error(sim_ctx *h) {
    int e[4];
    CU(cudaMemcpyAsync(e, h->d.err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (e[0] == SIM_EOVERFLOW) {
        char b[128];
        snprintf(b, sizeof b, "queue of link %d overflowed at step %d", e[1], e[2]);
        return fail(h, SIM_EOVERFLOW, b);
    }
    if (e[0]) return fail(h, e[0], "device error");
    return SIM_OK;
}

extern "C" int sim_reset(sim_handle h, int32_t T) {
    if (!h) return SIM_EINVAL;
    if (T < 1) return fail(h, SIM_EINVAL, "horizon must be >= 1");
    CU(cudaSetDevice(h->device));
    TRY(ensure_T(h, T));
    enqueue_reset(h, T);
    CU(cudaGetLastError());
    h->t = 0;
    h->T = T;
    h->n_bins = sim_n_bins(T, h->opt.obs_every);
    h->reset_done = true;
    return SIM_OK;
}

extern "C" int sim_step(sim_handle h, int32_t n_steps) {
    if (!h) return SIM_EINVAL;
    if (!h->reset_done) return fail(h, SIM_ESTATE, "sim_reset first");
    if (n_steps < 0 || h->t + n_steps > h->T) return fail(h, SIM_ESTATE, "step beyond the horizon");
    CU(cudaSetDevice(h->device));
    for (int k = 0; k < n_steps; ++k) {
        enqueue_step(h, h->t);
        h->t++;
        if (h->t == h->T) enqueue_obs_final(h, h->T);
    }
    CU(cudaGetLastError());
    return check_device_error(h);
}

static int copy_outputs(sim_ctx *h, sim_outputs *out) {
    if (!out) return SIM_OK;
    const int T = h->T, L = h->L;
    const size_t nb = (size_t)h->n_bins * L;
    const cudaMemcpyKind k = out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (out->counts) CU(cudaMemcpyAsync(out->counts, h->d.out_counts, nb * sizeof(int), k, h->stream));
    if (out->speed) CU(cudaMemcpyAsync(out->speed, h->d.out_speed, nb * sizeof(float), k, h->stream));
    if (out->travel_time) CU(cudaMemcpyAsync(out->travel_time, h->d.out_tt, nb * sizeof(float), k, h->stream));
    if (out->n_waiting || out->n_on || out->n_arrived) {
        std::vector<int> sd((size_t)4 * T);
        CU(cudaMemcpyAsync(sd.data(), h->d.step_delta, sd.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        std::vector<int64_t> nw(T + 1), non(T + 1), na(T + 1);
        nw[0] = h->N; non[0] = 0; na[0] = 0;
        for (int t = 0; t < T; ++t) {
            nw[t + 1] = nw[t] - sd[4 * t];
            na[t + 1] = na[t] + sd[4 * t + 1];
            non[t + 1] = h->N - nw[t + 1] - na[t + 1];
        }
        const std::vector<int64_t> *src[3] = {&nw, &non, &na};
        int64_t *dst[3] = {out->n_waiting, out->n_on, out->n_arrived};
        for (int a = 0; a < 3; ++a) {
            if (!dst[a]) continue;
            if (out->on_device)
                CU(cudaMemcpyAsync(dst[a], src[a]->data(), (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
            else
                memcpy(dst[a], src[a]->data(), (T + 1) * sizeof(int64_t));
        }
        if (out->on_device) CU(cudaStreamSynchronize(h->stream));
    }
    if (!out->on_device) CU(cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

extern "C" int sim_rollout(sim_handle h, int32_t T, sim_outputs *out) {
    if (!h) return SIM_EINVAL;
    if (T < 1) return fail(h, SIM_EINVAL, "horizon must be >= 1");
    CU(cudaSetDevice(h->device));
    TRY(ensure_T(h, T));
    auto it = h->graphs.find(T);
    if (it == h->graphs.end()) {
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_reset(h, T);
        for (int t = 0; t < T; ++t) enqueue_step(h, t);
        enqueue_obs_final(h, T);
        cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        if (ce != cudaSuccess) return fail(h, SIM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        cudaGraphExec_t ge;
        ce = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(h, SIM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        it = h->graphs.emplace(T, ge).first;
    }
    CU(cudaGraphLaunch(it->second, h->stream));
    h->t = T;
    h->T = T;
    h->n_bins = sim_n_bins(T, h->opt.obs_every);
    h->reset_done = true;
    TRY(copy_outputs(h, out));
    if (out && out->on_device) return SIM_OK;    // asynchronous: no host sync
    return check_device_error(h);
}

extern "C" int sim_step_counters(sim_handle h, int32_t *counters) {
    if (!h || !counters) return SIM_EINVAL;
    if (!h->reset_done) return fail(h, SIM_ESTATE, "no run");
    CU(cudaSetDevice(h->device));
    if (h->t > 0)
        CU(cudaMemcpyAsync(counters, h->d.step_delta, (size_t)4 * h->t * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

extern "C" int sim_profile_rollout(sim_handle h, int32_t T, sim_outputs *out, double *kernel_ms,
                                   int64_t *launches) {
    if (!h) return SIM_EINVAL;
    if (T < 1) return fail(h, SIM_EINVAL, "horizon must be >= 1");
    CU(cudaSetDevice(h->device));
    TRY(ensure_T(h, T));
    std::vector<cudaEvent_t> ev((size_t)4 * T + 2);
    for (auto &e : ev) CU(cudaEventCreate(&e));
    enqueue_reset(h, T);
    const int warps = h->L + (h->V + 31) / 32;
    for (int t = 0; t < T; ++t) {
        CU(cudaEventRecord(ev[4 * t + 0], h->stream));
        k_step_a<<<(warps * 32 + 127) / 128, 128, 0, h->stream>>>(h->d, t, 0);
        CU(cudaEventRecord(ev[4 * t + 1], h->stream));
        CU(cudaEventRecord(ev[4 * t + 2], h->stream));
        k_step_b<<<(h->L + h->V + 255) / 256, 256, 0, h->stream>>>(h->d, t);
        CU(cudaEventRecord(ev[4 * t + 3], h->stream));
    }
    CU(cudaEventRecord(ev[4 * T], h->stream));
    enqueue_obs_final(h, T);
    CU(cudaEventRecord(ev[4 * T + 1], h->stream));
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    double ms[3] = {0, 0, 0};
    for (int t = 0; t < T; ++t) {
        float a = 0, b = 0;
        CU(cudaEventElapsedTime(&a, ev[4 * t], ev[4 * t + 1]));
        CU(cudaEventElapsedTime(&b, ev[4 * t + 2], ev[4 * t + 3]));
        ms[0] += a;
        ms[1] += b;
    }
    float c = 0;
    CU(cudaEventElapsedTime(&c, ev[4 * T], ev[4 * T + 1]));
    ms[2] = c;
    for (auto &e : ev) cudaEventDestroy(e);
    if (kernel_ms) for (int k = 0; k < 3; ++k) kernel_ms[k] = ms[k];
    if (launches) { launches[0] = T; launches[1] = T; launches[2] = 1; }
    h->t = T;
    h->T = T;
    h->n_bins = sim_n_bins(T, h->opt.obs_every);
    h->reset_done = true;
    TRY(copy_outputs(h, out));
    return check_device_error(h);
}

extern "C" int sim_get_outputs(sim_handle h, sim_outputs *out) {
    if (!h || !out) return SIM_EINVAL;
    if (!h->reset_done) return fail(h, SIM_ESTATE, "no run");
    CU(cudaSetDevice(h->device));
    return copy_outputs(h, out);
}

extern "C" int sim_backward(sim_handle h, const float *, const float *, int32_t, sim_grads *) {
    if (!h) return SIM_EINVAL;
    return fail(h, SIM_ESTATE, "sim_backward: no recorded rollout");
}

extern "C" int sim_get_state(sim_handle h, sim_state_view *out) {
    if (!h || !out) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    const int L = h->L, N = h->N, V = h->V, S = h->S;
    std::vector<int4> lq(L);
    std::vector<float> pos(S);
    std::vector<int> svid(S), entry(N), vstate(N), fptr(V);
    CU(cudaMemcpyAsync(lq.data(), h->d.lq, L * sizeof(int4), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(pos.data(), (h->t & 1) ? h->d.pos1 : h->d.pos0, S * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(svid.data(), h->d.svid, S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(entry.data(), h->d.entry, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(vstate.data(), h->d.vstate, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(fptr.data(), h->d.fifo_ptr, V * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < N; ++i) {
        const int s = vstate[i] >= 0 ? -1 : vstate[i];
        if (out->veh_link) out->veh_link[i] = s;
        if (out->veh_pos) out->veh_pos[i] = 0.0;
        if (out->veh_rank) out->veh_rank[i] = -1;
        if (out->veh_entry) out->veh_entry[i] = entry[i];
    }
    for (int j = 0; j < L; ++j) {
        const int base = h->lst_host[4 * j], cap = h->lst_host[4 * j + 1];
        for (int k = 0; k < lq[j].y; ++k) {
            int idx = lq[j].x + k;
            if (idx >= cap) idx -= cap;
            const int v = svid[base + idx];
            if (v < 0 || v >= N) return fail(h, SIM_ESTATE, "corrupt queue");
            if (out->veh_link) out->veh_link[v] = j;
            if (out->veh_pos) out->veh_pos[v] = pos[base + idx];
            if (out->veh_rank) out->veh_rank[v] = k;
        }
        if (out->link_credit) out->link_credit[j] = lq[j].z;
        if (out->link_exits) out->link_exits[j] = lq[j].w;
    }
    if (out->fifo_off)
        for (int n = 0; n < V; ++n) out->fifo_off[n] = fptr[n] - h->fifo_beg[n];
    return SIM_OK;
}

extern "C" int sim_get_records(sim_handle h, sim_records *out) {
    if (!h || !out) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    const int L = h->L, V = h->V;
    std::vector<int> lc(L), lt(L), nc(V), nt(V);
    std::vector<unsigned long long> W(L);
    const int p = (h->t - 1) & 1;
    CU(cudaMemcpyAsync(lc.data(), h->d.cand_vid, L * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(lt.data(), h->d.cand_tgt, L * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(nc.data(), h->d.ncand_vid, V * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(nt.data(), h->d.ncand_tgt, V * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(W.data(), p ? h->d.W1 : h->d.W0, L * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < L; ++j) {
        if (out->link_cand) out->link_cand[j] = lt[j] == kTgtNone ? -1 : lc[j];
        if (out->link_target) out->link_target[j] = lt[j];
        if (out->link_in) out->link_in[j] = W[j] ? (int)(~(uint32_t)(W[j] & 0xffffffffull)) : -1;
    }
    for (int n = 0; n < V; ++n) {
        if (out->node_cand) out->node_cand[n] = nt[n] == kTgtNone ? -1 : nc[n];
        if (out->node_target) out->node_target[n] = nt[n];
    }
    return SIM_OK;
}

extern "C" int32_t sim_time(sim_handle h) { return h ? h->t : -1; }
extern "C" size_t sim_device_bytes(sim_handle h) { return h ? h->bytes : 0; }

extern "C" int sim_destroy(sim_handle h) {
    if (!h) return SIM_OK;
    release(h);
    delete h;
    return SIM_OK;
}

extern "C" const char *sim_last_error(sim_handle h) {
    return h ? h->err.c_str() : g_create_err.c_str();
}
