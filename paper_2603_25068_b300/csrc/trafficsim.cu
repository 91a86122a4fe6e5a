// trafficsim.cu -- host side of the simulator and the C ABI of include/trafficsim.h.
// Two forward executors run the same step:
//   * per-step kernels (ts_step.cuh): a rollout is captured once per horizon
//     into a CUDA graph of 2T + 2 kernels (reset, T x (k_step_a, k_step_b),
//     final observation); used when recording the reverse-pass tape and for
//     networks whose queues do not fit in shared memory;
//   * persistent (ts_persist.cuh): the whole run in one cooperative launch with
//     every queue resident in shared memory, one grid barrier per step.
#include "../../include/trafficsim.h"
#include "ts_backward.cuh"
#include "ts_persist.cuh"
#include "ts_batch.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <thread>
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
    const float4 geo = make_float4(L, udt, s, dtag);
    const_cast<float4 *>(d.geo)[j] = geo;
    // the bits k_step_a computes for a link with no vehicle (n = 0)
    const int va = vacant_after(0.0f, d.M, geo) ? 1 : 0, ar = arrives_after(0.0f, geo, d.M, d.eps_arr) ? 1 : 0;
    const_cast<int *>(d.ebits)[j] = 1 | (1 << 1) | (va << 2) | (va << 3) | (ar << 6) | (ar << 7);
    const_cast<float4 *>(d.tinfo)[j] = make_float4(a, g, __int_as_float(head[j]), __fmul_rn(L, 0.5f));
}

// The validity test of upload_params on parameters that live on the device:
// u, kappa, cost positive and finite, u dt below 2000 m, alpha, beta, w and the
// origin queues' merge priority finite; *perr becomes nonzero otherwise.
__global__ void k_check_params(const float *u, const float *kappa, const float *alpha, const float *beta,
                               const float *cost, const float *w, const float *alpha_origin, int L, int F, float dt,
                               int *perr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < L) {
        bad = !(u[i] > 0.0f) || !isfinite(u[i]) || !((double)u[i] * dt < 2000.0) || !(kappa[i] > 0.0f) ||
              !isfinite(kappa[i]) || !(cost[i] > 0.0f) || !isfinite(cost[i]) || !isfinite(alpha[i]) ||
              !isfinite(beta[i]);
    }
    if (i < F) bad = bad || !isfinite(w[i]);
    if (i == 0) bad = bad || !isfinite(*alpha_origin);
    if (bad) atomicOr(perr, 1);
}

__global__ void k_reset(DevSim d, const int *fifo_beg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.L) {
        const int4 st = d.lst[i];
        d.lq[i] = make_int4(0, 0, st.w, 0);
        d.vac[i] = kFlagVacant;
        d.W0[i] = 0ull;
        d.W1[i] = 0ull;
        d.lstat[i] = make_int4(0, 0, 0, 0);
        d.lpos[i] = make_longlong2(0, 0);
        d.crec[i] = make_int4(-1, kTgtNone, 0, 0);
    }
    if (i < d.V) { d.fifo_ptr[i] = fifo_beg[i]; d.nrec[i] = make_int2(-1, kTgtNone); }
    if (i < d.N) d.vstate[i] = kVehWaiting;
    if (i < 4) d.err[i] = 0;
}

// Vacancy / arrival flags of step t of every link from its queue at time t, as
// k_step_b selects them for an outcome without pop or push (set state).
__global__ void k_set_flags(DevSim d, int t) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.L) return;
    const int4 q = d.lq[j], st = d.lst[j];
    const float4 g = d.geo[j];
    const float *pc = (t & 1) ? d.pos1 : d.pos0;
    auto at = [&](int k) {
        int idx = q.x + k;
        if (idx >= st.y) idx -= st.y;
        return pc[st.x + idx];
    };
    const int n = q.y;
    const float M = d.M;
    const float xt = n >= 1 ? at(n - 1) : 0.0f, xpt = n >= 2 ? at(n - 2) : 0.0f, x0 = n >= 1 ? at(0) : 0.0f;
    const int vac = (n == 0 || vacant_after(xt, n >= 2 ? __fsub_rn(xpt, xt) : M, g)) ? 1 : 0;
    const int arr = (n >= 1 && arrives_after(x0, g, M, d.eps_arr)) ? 1 : 0;
    d.vac[j] = vac | (arr << 1);
}

// Choice-slot records (U, G, head, link) of every choice-set entry after a link
// and of every out-link of a node, from the per-link utility terms.
__global__ void k_choice_info(DevSim d, const int *lo_idx, int n_lo, const int *no_idx, int n_no) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_lo) {
        const int m = lo_idx[e];
        const float4 ti = d.tinfo[m];
        const_cast<float4 *>(d.loinfo)[e] = make_float4(ti.x, ti.y, ti.z, __int_as_float(m));
    }
    if (e < n_no) {
        const int m = no_idx[e];
        const float4 ti = d.tinfo[m];
        const_cast<float4 *>(d.noinfo)[e] = make_float4(ti.x, ti.y, ti.z, __int_as_float(m));
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------

struct sim_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // reverse pass: the merge/choice Jacobian kernel runs on a second stream
    cudaStream_t jstream = nullptr;
    cudaEvent_t ev_z = nullptr, ev_g = nullptr;
    // ... and the segment recomputation on a third stream, double-buffered tape;
    // the reverse kernels themselves on a high-priority stream
    cudaStream_t rstream = nullptr, vstream = nullptr;
    int recompute = SIM_RECOMPUTE_SERIAL;
    cudaEvent_t ev_r[2] = {nullptr, nullptr}, ev_b[2] = {nullptr, nullptr};
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
    int *d_lo_idx = nullptr, *d_no_idx = nullptr;
    int n_lo = 0, n_no = 0;
    int stage = 4096;                    // queue slots staged per link block
    int stage_max = 0;                   // largest staged slot count of a block
    int *d_blk = nullptr;
    int cap_blk = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
    // run state
    int t = 0, T = 0, n_bins = 0;
    bool reset_done = false;
    int *d_perr = nullptr;               // set by k_check_params when device parameters are invalid
    int cap_T = 0;                       // capacity of the per-T output buffers
    std::map<int, cudaGraphExec_t> graphs;
    std::string err;
    // reverse mode (options.ckpt_every > 0)
    int K = 0;                           // steps per checkpoint segment
    int route_cap = 0;
    bool tape_ready = false;             // last call was a recorded sim_rollout
    int bmode = 2;                       // batch mode (running / closing last bin / idle)
    int cap_seg = 0;                     // checkpoints allocated
    BwdDev b{};
    struct Ckpt {
        int4 *lq = nullptr, *lstat = nullptr;
        int *vac = nullptr, *sentry = nullptr, *fifo = nullptr, *vstate = nullptr;
        float *pos = nullptr;
        int2 *saux = nullptr;
        longlong2 *lpos = nullptr;
    } ck;
    int *d_dummy = nullptr;              // step counters of recomputed steps
    int *d_od = nullptr;
    float *d_od_lambda = nullptr;
    // persistent executor
    std::vector<int> lo_count;           // choice-set size after each link
    std::vector<int> no_ptr_host;        // out-links of each node (CSR offsets)
    int executor = SIM_EXEC_AUTO;        // requested
    int bar_extra = 0;                   // test hook: missing arrivals at the next launch's barriers
    bool persist_ok = false;             // the network fits (groups, shared memory, co-residency)
    std::string persist_why;             // reason when it does not
    int G = 0;                           // CTAs (one per SM at most)
    std::vector<long long> pw;           // partition weights (empty: queue capacity + 16)
    int *d_grp = nullptr;                // group bounds, one slot per SM + 1
    size_t persist_smem = 0;
    PArgs pa{};
};

// Workspace of the reverse pass (tape of one segment, adjoints, accumulators),
// shared by every handle of a device: sim_backward holds the device's lock for
// the whole call, grows the workspace when a handle needs more and returns only
// after its stream has drained.  It is released when the process exits.
// Reverse-pass workspaces of a device: a call takes a free one large enough
// (growing or adding one if none is), so reverse passes of different
// simulators can run at the same time; freed workspaces stay for reuse.
struct BwdWs {
    void *buf = nullptr;
    size_t cap = 0;
    bool busy = false;
};
struct BwdPool {
    std::mutex mu;
    std::vector<BwdWs *> ws;
};
static BwdPool g_bwd_pool[64];

static BwdWs *bwd_take(int device, size_t need) {
    BwdPool &pool = g_bwd_pool[device];
    std::lock_guard<std::mutex> lock(pool.mu);
    BwdWs *fit = nullptr, *any = nullptr;
    for (BwdWs *w : pool.ws) {
        if (w->busy) continue;
        if (w->cap >= need && (!fit || w->cap < fit->cap)) fit = w;
        if (!any || w->cap > any->cap) any = w;
    }
    BwdWs *w = fit ? fit : any;
    if (!w) {
        w = new BwdWs();
        pool.ws.push_back(w);
    }
    w->busy = true;
    return w;
}

// Gives the workspace back when the call ends, once the streams that may use
// it have drained (an error can end the call with work in flight).
struct BwdLease {
    BwdPool *pool;
    BwdWs *w;
    std::vector<cudaStream_t> streams;
    ~BwdLease() {
        for (cudaStream_t s : streams)
            if (s) cudaStreamSynchronize(s);
        std::lock_guard<std::mutex> lock(pool->mu);
        w->busy = false;
    }
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

// Device memory of simulators and batches comes from one memory pool per
// device, allocated and freed in stream order: releasing a simulator does not
// wait for the whole device (as cudaFree does), and the next simulator reuses
// the freed blocks without new mappings.  Like a caching allocator, the pool
// keeps what it has mapped (up to the largest working set) until the process
// ends or sim_release_cached_memory is called.
static std::mutex g_mpool_mu;
static cudaMemPool_t g_mpool[64];

static cudaError_t pool_alloc(void **p, size_t bytes, int device, cudaStream_t s) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_mpool_mu);
        if (!g_mpool[device]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            cudaError_t e = cudaMemPoolCreate(&g_mpool[device], &props);
            if (e != cudaSuccess) { g_mpool[device] = nullptr; return e; }
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(g_mpool[device], cudaMemPoolAttrReleaseThreshold, &keep);
            // never make an allocating stream wait for the work of the stream
            // that freed a block (serving creates simulators beside a busy
            // batch): reuse a block only once its free has completed
            int no = 0;
            cudaMemPoolSetAttribute(g_mpool[device], cudaMemPoolReuseAllowInternalDependencies, &no);
        }
        pool = g_mpool[device];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

extern "C" int sim_release_cached_memory(int32_t device) {
    if (device < 0 || device >= 64) return SIM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SIM_ECUDA;
    {                                    // idle reverse-pass workspaces
        BwdPool &pool = g_bwd_pool[device];
        std::lock_guard<std::mutex> lock(pool.mu);
        std::vector<BwdWs *> keep;
        for (BwdWs *w : pool.ws) {
            if (w->busy) { keep.push_back(w); continue; }
            if (w->buf) cudaFreeAsync(w->buf, nullptr);
            delete w;
        }
        pool.ws = keep;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return SIM_ECUDA;
    std::lock_guard<std::mutex> lock(g_mpool_mu);
    if (g_mpool[device] && cudaMemPoolTrimTo(g_mpool[device], 0) != cudaSuccess) return SIM_ECUDA;
    return SIM_OK;
}

template <class T>
static int dalloc(sim_ctx *h, T **p, size_t n) {
    void *q = nullptr;
    size_t b = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = pool_alloc(&q, b, h->device, h->stream);
    if (e != cudaSuccess) return fail(h, SIM_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
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

// The dynamic shared-memory limit is an attribute of a kernel function, shared by
// every handle: raise it monotonically (per device) to the largest size needed.
static std::mutex g_attr_mu;
static size_t g_attr_a[64], g_attr_at[64], g_attr_ba[64];

template <class K>
static cudaError_t raise_smem_attr(K kernel, size_t *cur, int device, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (bytes <= cur[device]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur[device] = bytes;
    return e;
}

// Pack consecutive links into link blocks of k_step_a: at most kLinksPerBlock
// links whose queue capacities add up to at most `stage` slots (a larger link
// gets a block of its own).
static int build_blocks(sim_ctx *h) {
    std::vector<int> blk{0};
    int slots = 0, nl = 0, smax = 0;
    for (int j = 0; j < h->L; ++j) {
        const int cap = h->lst_host[4 * j + 1];
        if (nl > 0 && (nl == kLinksPerBlock || slots + cap > h->stage)) {
            blk.push_back(j);
            smax = std::max(smax, slots);
            slots = 0;
            nl = 0;
        }
        slots += cap;
        nl += 1;
    }
    blk.push_back(h->L);
    smax = std::max(smax, slots);
    // origin queues are spread over the blocks, at most kNodesPerBlock each
    const int nlink_blocks = (int)blk.size() - 1;
    const int nblk = std::max(nlink_blocks, (h->V + kNodesPerBlock - 1) / kNodesPerBlock);
    while ((int)blk.size() < nblk + 1) blk.push_back(h->L);
    if (!h->d_blk || h->cap_blk < (int)blk.size()) {
        h->cap_blk = std::max((int)blk.size(), h->L + 1);
        TRY(dalloc(h, &h->d_blk, (size_t)h->cap_blk));
    }
    CU(cudaMemcpyAsync(h->d_blk, blk.data(), blk.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->d.blk_links = h->d_blk;
    h->d.nblk = nblk;
    h->d.npb = (h->V + nblk - 1) / nblk;
    h->stage_max = smax;
    CU(raise_smem_attr(k_step_a, g_attr_a, h->device, (size_t)smax * sizeof(float)));
    CU(raise_smem_attr(k_step_a_tape, g_attr_at, h->device, (size_t)smax * sizeof(float)));
    return SIM_OK;
}

// Groups of the persistent executor: consecutive links packed into at most one
// group per SM, each within kPLinks links and the shared memory left for queue
// slots, with the largest group weight made as small as possible (binary search
// over the bound, greedy packing).  A link weighs its queue capacity + 16 slots,
// or the weight set by sim_set_partition_weights.
static size_t g_attr_p[64], g_attr_pt[64];
static int build_groups(sim_ctx *h) {
    h->persist_ok = false;
    int nsm = 0, optin = 0;
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const long long budget = (long long)optin - (long long)sizeof(PSmem);
    const int L = h->L, V = h->V;
    // shared-memory bytes of a link: its ring slots and its staged choice records
    std::vector<long long> cap(L), lob(L);
    long long wsum = 0, wmax = 0;
    for (int j = 0; j < L; ++j) {
        cap[j] = h->lst_host[4 * j + 1];
        lob[j] = 4 * cap[j] + 16 * (long long)h->lo_count[j];
    }
    auto weight = [&](int j) { return h->pw.empty() ? cap[j] + 16 : h->pw[j]; };
    for (int j = 0; j < L; ++j) {
        wsum += weight(j);
        wmax = std::max(wmax, weight(j));
    }
    // the origin queues of a group are the nodes [g npg, (g + 1) npg)
    auto node_bytes = [&](int G) {
        const int npg = (V + G - 1) / G;
        long long worst = 0;
        for (int g = 0; g < G; ++g) {
            const int n0 = std::min(V, g * npg), n1 = std::min(V, (g + 1) * npg);
            worst = std::max(worst, 16LL * (h->no_ptr_host[n1] - h->no_ptr_host[n0]));
        }
        return worst;
    };
    long long reserve = node_bytes(std::max(1, std::min(nsm, (V + kPNodes - 1) / kPNodes)));
    std::vector<int> starts;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const long long lbud = budget - reserve - 16;
        bool fits = true;
        for (int j = 0; j < L; ++j) fits = fits && lob[j] <= lbud;
        if (!fits) {
            h->persist_why = "a link queue is larger than the shared memory of one CTA";
            return SIM_OK;
        }
        auto pack = [&](long long bound, std::vector<int> *out) {
            int groups = 0, nl = 0;
            long long w = 0, bytes = 0;
            if (out) out->clear();
            for (int j = 0; j < L; ++j) {
                const long long wj = weight(j);
                if (nl == 0 || nl == kPLinks || w + wj > bound || bytes + lob[j] > lbud) {
                    if (out) out->push_back(j);
                    ++groups;
                    nl = 0; w = 0; bytes = 0;
                }
                ++nl; w += wj; bytes += lob[j];
            }
            return groups;
        };
        long long lo = std::max(wmax, (wsum + nsm - 1) / nsm), hi = std::max(lo, wsum);
        if (pack(hi, nullptr) > nsm) {
            h->persist_why = "the queues do not fit in the shared memory of the GPU";
            return SIM_OK;
        }
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (pack(mid, nullptr) <= nsm) hi = mid; else lo = mid + 1;
        }
        pack(lo, &starts);
        const int G = std::max((int)starts.size(), (V + kPNodes - 1) / kPNodes);
        const long long need = node_bytes(G);
        if (need <= reserve) break;
        if (attempt == 1) {
            h->persist_why = "the origin nodes' out-links do not fit in shared memory";
            return SIM_OK;
        }
        reserve = need;
    }
    const int G = std::max((int)starts.size(), (V + kPNodes - 1) / kPNodes);
    if (G > nsm) {
        h->persist_why = "too many origin nodes for one CTA per SM";
        return SIM_OK;
    }
    std::vector<int> grp(starts);
    grp.push_back(L);
    while ((int)grp.size() < G + 1) grp.push_back(L);
    const int npg = (V + G - 1) / G;
    size_t dmax = 0;
    for (int g = 0; g < G; ++g) {
        long long sl = 0, nlo = 0;
        for (int j = grp[g]; j < grp[g + 1]; ++j) { sl += cap[j]; nlo += h->lo_count[j]; }
        const int n0 = std::min(V, g * npg), n1 = std::min(V, (g + 1) * npg);
        dmax = std::max(dmax, p_dyn_bytes(sl, nlo, h->no_ptr_host[n1] - h->no_ptr_host[n0]));
    }
    const size_t smem = sizeof(PSmem) + dmax;
    if (smem > (size_t)optin) {
        h->persist_why = "a group does not fit in the shared memory of one CTA";
        return SIM_OK;
    }
    CU(raise_smem_attr(k_persist, g_attr_p, h->device, smem));
    CU(raise_smem_attr(k_persist_tape, g_attr_pt, h->device, smem));
    int per_sm = 0, per_sm_t = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPT, smem));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_t, k_persist_tape, kPT, smem));
    per_sm = std::min(per_sm, per_sm_t);
    if (per_sm < 1 || G > per_sm * nsm) {
        h->persist_why = "the CTAs cannot all be resident at once";
        return SIM_OK;
    }
    if (!h->d_grp) TRY(dalloc(h, &h->d_grp, (size_t)nsm + 1));
    CU(cudaMemcpyAsync(h->d_grp, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (!h->pa.W3) {
        TRY(dalloc(h, &h->pa.W3, (size_t)3 * L));
        TRY(dalloc(h, &h->pa.bar, 4));
    }
    h->pa.grp_links = h->d_grp;
    h->pa.npg = npg;
    h->pa.packz = (h->N < (1 << 24) && h->Z <= 256) ? 1 : 0;
    h->G = G;
    h->persist_smem = smem;
    h->persist_ok = true;
    return SIM_OK;
}

// persistent executor in use for the next forward run of this handle (also the
// checkpointed forward of handles that record the reverse-pass tape and their
// segment recomputation)
static bool use_persist(const sim_ctx *h) { return h->persist_ok && h->executor != SIM_EXEC_STEP; }

// steps [t0, t1) (+ the observation-only pass at t1) in one cooperative launch
// of d (tape: the recording kernel, d's tape pointers the bases of record 0)
static int enqueue_persist_d(sim_ctx *h, const DevSim &d, int t0, int t1, int final_obs, bool tape,
                             cudaStream_t st = nullptr) {
    if (!st) st = h->stream;
    PArgs a = h->pa;
    a.t0 = t0;
    a.t1 = t1;
    a.final_obs = final_obs;
    a.S = h->S;
    a.bar_extra = h->bar_extra;
    h->bar_extra = 0;
    // barrier-wait car-following over queue positions >= 2 only: on networks
    // with 8 or more vehicles per link, whose queues are long enough for it
    a.skip2 = (long long)h->N >= 8LL * h->L ? 1 : 0;
    for (int r = 0; r < 10; ++r) {               // the Philox key schedule of d's keys
        a.rk[0][r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[1][r] = d.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    CU(cudaMemsetAsync(a.W3, 0, (size_t)3 * h->L * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(a.bar, 0, sizeof(unsigned), st));
    DevSim dd = d;
    void *args[2] = {(void *)&dd, (void *)&a};
    CU(cudaLaunchCooperativeKernel(tape ? (const void *)k_persist_tape : (const void *)k_persist, dim3(h->G), dim3(kPT),
                                   args, h->persist_smem, st));
    return SIM_OK;
}
static int enqueue_persist(sim_ctx *h, int t0, int t1, int final_obs) {
    return enqueue_persist_d(h, h->d, t0, t1, final_obs, false);
}

static int upload_params(sim_ctx *h, const sim_params *par) {
    const int L = h->L, F = h->F;
    if (!par->u || !par->kappa || !par->alpha || !par->beta || !par->cost || (F > 0 && !par->w))
        return fail(h, SIM_EINVAL, "null parameter array");
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
    if (h->d_perr) CU(cudaMemsetAsync(h->d_perr, 0, sizeof(int), h->stream));
    k_params<<<(L + 255) / 256, 256, 0, h->stream>>>(h->d, h->d_len, h->d_u, h->d_kappa, h->d_beta, h->d_cost,
                                                     h->d_phi, h->d_psi, h->d_w, h->d_head, h->opt.dn,
                                                     h->opt.eps_tag);
    const int ne = std::max(h->n_lo, h->n_no);
    k_choice_info<<<(ne + 255) / 256, 256, 0, h->stream>>>(h->d, h->d_lo_idx, h->n_lo, h->d_no_idx, h->n_no);
    CU(cudaGetLastError());
    // the captured graphs read the parameters from device memory and stay valid;
    // host copies of the parameters must outlive the asynchronous uploads
    CU(cudaStreamSynchronize(h->stream));
    h->reset_done = false;
    return SIM_OK;
}

// ---- host set-up on several threads ----
// f(t, T) on threads t = 0 .. T - 1 (the calling thread is t = 0)
template <class F>
static void host_parallel(int T, F f) {
    if (T <= 1) { f(0, 1); return; }
    std::vector<std::thread> th;
    th.reserve(T - 1);
    for (int t = 1; t < T; ++t) th.emplace_back(f, t, T);
    f(0, T);
    for (auto &x : th) x.join();
}
static int host_threads(size_t n) {
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    return (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(hw, 8), n / 65536));
}
// Stable counting sort of n records by key(r) in [0, K) from in to out, on T
// threads: per-thread counts over contiguous chunks, offsets in (key, thread)
// order, then each thread scatters its chunk in order.
template <class R, class Key>
static void counting_sort(const R *in, R *out, size_t n, size_t K, Key key, int T) {
    std::vector<size_t> cnt((size_t)T * K, 0);
    host_parallel(T, [&](int t, int nt) {
        size_t *c = &cnt[(size_t)t * K];
        for (size_t i = n * t / nt, e = n * (t + 1) / nt; i < e; ++i) c[key(in[i])]++;
    });
    size_t run = 0;
    for (size_t k = 0; k < K; ++k)
        for (int t = 0; t < T; ++t) {
            const size_t c = cnt[(size_t)t * K + k];
            cnt[(size_t)t * K + k] = run;
            run += c;
        }
    host_parallel(T, [&](int t, int nt) {
        size_t *c = &cnt[(size_t)t * K];
        for (size_t i = n * t / nt, e = n * (t + 1) / nt; i < e; ++i) out[c[key(in[i])]++] = in[i];
    });
}

static int create_impl(sim_ctx *h, const sim_network *net, const sim_demand *dem, const sim_params *par,
                       const sim_options *opt) {
    if (!net || !dem || !par || !opt) return fail(h, SIM_EINVAL, "null argument");
    const int V = net->V, L = net->L, N = dem->N, F = net->F, Z = net->Z;
    if (V <= 0 || L <= 0 || N < 0 || F < 0 || Z <= 0) return fail(h, SIM_EINVAL, "bad sizes");
    if (!net->tail || !net->head || !net->length || !net->q_fx || !net->node_zone || !net->dest_feat ||
        (F > 0 && (!net->phi || !net->psi)) || !par->u)
        return fail(h, SIM_EINVAL, "null network array");
    if (N > 0 && (!dem->origin || !dem->dest_zone || !dem->dep_step))
        return fail(h, SIM_EINVAL, "null demand array");
    if (!(opt->dt > 0) || !(opt->dn > 0) || opt->obs_every <= 0 || !(opt->tau_gumbel > 0))
        return fail(h, SIM_EINVAL, "bad options");
    for (int j = 0; j < L; ++j)
        if (!((double)par->u[j] * opt->dt < 2000.0)) return fail(h, SIM_EINVAL, "u dt must be below 2000 m");
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
    h->lo_count.resize(L);
    for (int l = 0; l < L; ++l) h->lo_count[l] = lnode[4 * l + 3] - lnode[4 * l + 2];
    h->no_ptr_host = no_ptr;
    h->S = (int)S;
    h->lst_host = lst;
    // origin queues: vehicles ordered by (origin, departure step, id), as two
    // stable counting sorts -- by departure step over the ids, then by origin
    // -- that move whole records (id, origin, departure step, destination
    // zone), so that neither pass gathers from the demand arrays at random;
    // both run on several host threads
    struct VRec { int id, origin, dep, zone; };
    std::vector<int> fifo(N), fifo_beg(V + 1, 0), fifo_dep(N), fifo_aux(2 * (size_t)N);
    {
        const int T = host_threads((size_t)N);
        std::unique_ptr<VRec[]> rec(new VRec[std::max(N, 1)]), tmp(new VRec[std::max(N, 1)]);
        int max_dep = 0;
        for (int i = 0; i < N; ++i) max_dep = std::max(max_dep, dem->dep_step[i]);
        host_parallel(T, [&](int t, int nt) {
            for (size_t i = (size_t)N * t / nt, e = (size_t)N * (t + 1) / nt; i < e; ++i)
                rec[i] = VRec{(int)i, dem->origin[i], dem->dep_step[i], dem->dest_zone[i]};
        });
        if (max_dep < (1 << 24)) {
            counting_sort(rec.get(), tmp.get(), (size_t)N, (size_t)max_dep + 1, [](const VRec &r) { return (size_t)r.dep; }, T);
        } else {                         // departure steps too far apart for counting
            std::copy(rec.get(), rec.get() + N, tmp.get());
            std::stable_sort(tmp.get(), tmp.get() + N, [](const VRec &a, const VRec &b) { return a.dep < b.dep; });
        }
        counting_sort(tmp.get(), rec.get(), (size_t)N, (size_t)V, [](const VRec &r) { return (size_t)r.origin; }, T);
        for (int i = 0; i < N; ++i) fifo_beg[dem->origin[i] + 1]++;
        for (int n = 0; n < V; ++n) fifo_beg[n + 1] += fifo_beg[n];
        host_parallel(T, [&](int t, int nt) {
            for (size_t k = (size_t)N * t / nt, e = (size_t)N * (t + 1) / nt; k < e; ++k) {
                const VRec r = rec[k];
                fifo[k] = r.id;
                fifo_dep[k] = r.dep;
                fifo_aux[2 * k] = r.id;
                fifo_aux[2 * k + 1] = r.zone;
            }
        });
    }
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
    int *ebits_d;
    TRY(dalloc(h, &ebits_d, L)); d.ebits = ebits_d;
    TRY(dalloc(h, &tinfo, L)); d.tinfo = tinfo;
    TRY(upload(h, &lstd, (const int4 *)lst.data(), L)); d.lst = lstd;
    TRY(upload(h, &lnoded, (const int4 *)lnode.data(), L)); d.lnode = lnoded;
    float *alpha_d;
    TRY(dalloc(h, &alpha_d, L + 1)); d.alpha = alpha_d;     // [L] = origin queues
    int *p;
    TRY(upload(h, &h->d_lo_idx, lo_idx.data(), lo_idx.size()));
    TRY(upload(h, &p, no_ptr.data(), no_ptr.size())); d.no_ptr = p;
    TRY(upload(h, &h->d_no_idx, no_idx.data(), no_idx.size()));
    h->n_lo = (int)lo_idx.size();
    h->n_no = (int)no_idx.size();
    float4 *lo_info, *no_info;
    TRY(dalloc(h, &lo_info, lo_idx.size())); d.loinfo = lo_info;
    TRY(dalloc(h, &no_info, no_idx.size())); d.noinfo = no_info;
    TRY(upload(h, &p, net->node_zone, V)); d.node_zone = p;
    TRY(upload(h, &p, fifo_end.data(), V)); d.fifo_end = p;
    int2 *fa;
    TRY(upload(h, &fa, (const int2 *)fifo_aux.data(), N)); d.fifo_list = fa;
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
    TRY(dalloc(h, &d.saux, S));
    TRY(dalloc(h, &d.sentry, S));
    TRY(dalloc(h, &d.W0, L));
    TRY(dalloc(h, &d.W1, L));
    TRY(dalloc(h, &d.crec, L));
    TRY(dalloc(h, &d.nrec, V));
    TRY(dalloc(h, &d.fifo_ptr, V));
    TRY(dalloc(h, &d.vstate, N));
    TRY(dalloc(h, &d.lstat, L));
    TRY(dalloc(h, &d.lpos, L));
    TRY(dalloc(h, &d.err, 4));
    TRY(dalloc(h, &h->d_perr, 1));
    CU(cudaMemsetAsync(h->d_perr, 0, sizeof(int), h->stream));
    CU(cudaMemsetAsync(d.err, 0, 4 * sizeof(int), h->stream));
    CU(cudaMemsetAsync(d.pos0, 0, (size_t)S * sizeof(float), h->stream));
    CU(cudaMemsetAsync(d.pos1, 0, (size_t)S * sizeof(float), h->stream));
    CU(cudaMemsetAsync(d.saux, 0xff, (size_t)S * sizeof(int2), h->stream));
    CU(cudaMemsetAsync(d.sentry, 0, (size_t)S * sizeof(int), h->stream));
    d.tag_tape = nullptr;
    d.route_log = nullptr;
    d.route_len = nullptr;
    d.route_cap = 0;
    if (opt->ckpt_every > 0) {
        if (opt->route_cap <= 0) return fail(h, SIM_EINVAL, "route_cap must be positive with ckpt_every > 0");
        h->K = opt->ckpt_every;
        h->route_cap = (opt->route_cap + 7) & ~7;     // rows of 64-byte multiples: 16-byte loads in the reverse pass
        const int K = h->K;
        BwdDev &b = h->b;
        b.S = (int)S; b.K = K; b.cap = h->route_cap; b.n_od = dem->n_od;
        b.tau = opt->tau_gumbel;
        b.inv_tau = 1.0 / (double)opt->tau_gumbel;
        TRY(dalloc(h, &d.route_log, (size_t)N * h->route_cap));
        TRY(dalloc(h, &d.route_len, N));
        d.route_cap = h->route_cap;
        b.route_log = d.route_log;
        b.route_len = d.route_len;
        if ((N > 0 && !dem->od) || (dem->n_od > 0 && !dem->od_lambda))
            return fail(h, SIM_EINVAL, "null od / od_lambda array");
        TRY(upload(h, &h->d_od, dem->od, N));
        TRY(upload(h, &h->d_od_lambda, dem->od_lambda, std::max(dem->n_od, 1)));
        for (int k = 0; k < dem->n_od; ++k)
            if (!(dem->od_lambda[k] > 0.0f)) return fail(h, SIM_EINVAL, "od_lambda must be positive");
        for (int i = 0; i < N; ++i)
            if (dem->od[i] < 0 || dem->od[i] >= dem->n_od) return fail(h, SIM_EINVAL, "od out of range");
        b.od = h->d_od;
        b.od_lambda = h->d_od_lambda;
    }
    TRY(build_blocks(h));
    TRY(build_groups(h));
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
    for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
    h->allocs.clear();
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
    if (h->jstream) cudaStreamSynchronize(h->jstream);
    if (h->rstream) cudaStreamSynchronize(h->rstream);
    for (cudaEvent_t e : {h->ev_z, h->ev_g, h->ev_r[0], h->ev_r[1], h->ev_b[0], h->ev_b[1]})
        if (e) cudaEventDestroy(e);
    if (h->vstream) cudaStreamSynchronize(h->vstream);
    if (h->jstream) cudaStreamDestroy(h->jstream);
    if (h->rstream) cudaStreamDestroy(h->rstream);
    if (h->vstream) cudaStreamDestroy(h->vstream);
    h->jstream = h->rstream = h->vstream = nullptr;
    h->ev_z = h->ev_g = nullptr;
    h->ev_r[0] = h->ev_r[1] = h->ev_b[0] = h->ev_b[1] = nullptr;
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

extern "C" int sim_set_params_device(sim_handle h, const sim_params *par, const float *alpha_origin) {
    if (!h || !par || !alpha_origin) return SIM_EINVAL;
    const int L = h->L, F = h->F;
    if (!par->u || !par->kappa || !par->alpha || !par->beta || !par->cost || (F > 0 && !par->w))
        return fail(h, SIM_EINVAL, "null parameter array");
    CU(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    CU(cudaMemsetAsync(h->d_perr, 0, sizeof(int), s));
    const int nc = std::max(std::max(L, F), 1);
    k_check_params<<<(nc + 255) / 256, 256, 0, s>>>(par->u, par->kappa, par->alpha, par->beta, par->cost,
                                                   F > 0 ? par->w : par->u, alpha_origin, L, F, h->opt.dt,
                                                   h->d_perr);
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    CU(cudaMemcpyAsync(h->d_u, par->u, L * sizeof(float), k, s));
    CU(cudaMemcpyAsync(h->d_kappa, par->kappa, L * sizeof(float), k, s));
    CU(cudaMemcpyAsync(const_cast<float *>(h->d.alpha), par->alpha, L * sizeof(float), k, s));
    CU(cudaMemcpyAsync(const_cast<float *>(h->d.alpha) + L, alpha_origin, sizeof(float), k, s));
    CU(cudaMemcpyAsync(h->d_beta, par->beta, L * sizeof(float), k, s));
    CU(cudaMemcpyAsync(h->d_cost, par->cost, L * sizeof(float), k, s));
    if (F) CU(cudaMemcpyAsync(h->d_w, par->w, F * sizeof(float), k, s));
    k_params<<<(L + 255) / 256, 256, 0, s>>>(h->d, h->d_len, h->d_u, h->d_kappa, h->d_beta, h->d_cost, h->d_phi,
                                             h->d_psi, h->d_w, h->d_head, h->opt.dn, h->opt.eps_tag);
    const int ne = std::max(h->n_lo, h->n_no);
    k_choice_info<<<(ne + 255) / 256, 256, 0, s>>>(h->d, h->d_lo_idx, h->n_lo, h->d_no_idx, h->n_no);
    CU(cudaGetLastError());
    h->reset_done = false;
    return SIM_OK;
}

// per-horizon buffers: outputs and step counters
static int ensure_T(sim_ctx *h, int T) {
    if (T <= h->cap_T) return SIM_OK;
    const int nb = sim_n_bins(T, h->opt.obs_every);
    // outputs are re-pointed: cached graphs bake the old pointers
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
    h->graphs.clear();
    TRY(dalloc(h, &h->d.out_counts, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.out_speed, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.out_tt, (size_t)nb * h->L));
    TRY(dalloc(h, &h->d.step_delta, (size_t)4 * T));
    if (h->K > 0) {
        TRY(dalloc(h, &h->d_dummy, (size_t)4 * T));
        const int nseg = (T + h->K - 1) / h->K;
        if (nseg > h->cap_seg) {
            const size_t L = h->L, S = h->S, V = h->V, N = h->N;
            TRY(dalloc(h, &h->ck.lq, nseg * L)); TRY(dalloc(h, &h->ck.lstat, nseg * L));
            TRY(dalloc(h, &h->ck.vac, nseg * L)); TRY(dalloc(h, &h->ck.sentry, nseg * S));
            TRY(dalloc(h, &h->ck.fifo, nseg * V)); TRY(dalloc(h, &h->ck.vstate, nseg * N));
            TRY(dalloc(h, &h->ck.pos, nseg * S)); TRY(dalloc(h, &h->ck.saux, nseg * S));
            TRY(dalloc(h, &h->ck.lpos, nseg * L));
            h->cap_seg = nseg;
        }
    }
    h->cap_T = T;
    return SIM_OK;
}

// checkpoint s <-> dynamic state at the start of step s K (positions in buffer
// (s K) & 1), one launch
static void ckpt_copy(sim_ctx *h, int s, bool save, cudaStream_t st = nullptr) {
    if (!st) st = h->stream;
    CkDev c{};
    c.K = h->K; c.L = h->L; c.S = h->S; c.V = h->V; c.N = h->N;
    c.lq = h->ck.lq; c.lstat = h->ck.lstat; c.vac = h->ck.vac; c.sentry = h->ck.sentry; c.fifo = h->ck.fifo;
    c.vstate = h->ck.vstate; c.pos = h->ck.pos; c.saux = h->ck.saux; c.lpos = h->ck.lpos;
    const size_t n = std::max(std::max((size_t)h->S, (size_t)h->N), std::max((size_t)h->L, (size_t)h->V));
    const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    k_ckpt<<<grid, 256, 0, st>>>(h->d, c, s * h->K, save ? 1 : 0);
}

static void enqueue_reset(sim_ctx *h, int T) {
    const int nmax = std::max(std::max(h->L, h->V), std::max(h->N, 4));
    cudaMemsetAsync(h->d.step_delta, 0, (size_t)4 * T * sizeof(int), h->stream);
    const int nb = sim_n_bins(T, h->opt.obs_every);
    cudaMemsetAsync(h->d.out_counts, 0, (size_t)nb * h->L * sizeof(int), h->stream);
    k_reset<<<(nmax + 255) / 256, 256, 0, h->stream>>>(h->d, h->d_fifo_beg);
    if (h->d.route_len) cudaMemsetAsync(h->d.route_len, 0, (size_t)h->N * sizeof(int), h->stream);
}

static void enqueue_a(sim_ctx *h, int t, int obs_only) {
    const size_t smem = (size_t)h->stage_max * sizeof(float);
    k_step_a<<<h->d.nblk, kBlockA, smem, h->stream>>>(h->d, t, obs_only);
}

static void enqueue_b(sim_ctx *h, int t) {
    k_step_b<<<(h->L + h->V + 255) / 256, 256, 0, h->stream>>>(h->d, t);
}

static void enqueue_step(sim_ctx *h, int t) {
    enqueue_a(h, t, 0);
    enqueue_b(h, t);
}

static void enqueue_obs_final(sim_ctx *h, int T) { enqueue_a(h, T, 1); }

static int check_device_error(sim_ctx *h) {
    int e[4], perr = 0;
    CU(cudaMemcpyAsync(e, h->d.err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(&perr, h->d_perr, sizeof perr, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (perr) return fail(h, SIM_EINVAL, "invalid parameter (checked on the device by sim_set_params_device)");
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
    h->tape_ready = false;
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
    if (use_persist(h) && h->K == 0 && n_steps > 0) {
        const int t1 = h->t + n_steps;
        TRY(enqueue_persist(h, h->t, t1, t1 == h->T));
        h->t = t1;
    } else {
        for (int k = 0; k < n_steps; ++k) {
            enqueue_step(h, h->t);
            h->t++;
            if (h->t == h->T) enqueue_obs_final(h, h->T);
        }
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
    if (use_persist(h)) {
        enqueue_reset(h, T);
        if (h->K > 0) {              // one launch per checkpoint segment, the state saved before each
            for (int t0 = 0; t0 < T; t0 += h->K) {
                const int t1 = std::min(T, t0 + h->K);
                ckpt_copy(h, t0 / h->K, true);
                TRY(enqueue_persist(h, t0, t1, t1 == T));
            }
        } else {
            TRY(enqueue_persist(h, 0, T, 1));
        }
        CU(cudaGetLastError());
        h->t = T;
        h->T = T;
        h->n_bins = sim_n_bins(T, h->opt.obs_every);
        h->reset_done = true;
        h->tape_ready = h->K > 0;
        TRY(copy_outputs(h, out));
        if (out && out->on_device) return SIM_OK;
        return check_device_error(h);
    }
    auto it = h->graphs.find(T);
    if (it == h->graphs.end()) {
        cudaGraph_t g;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_reset(h, T);
        for (int t = 0; t < T; ++t) {
            if (h->K > 0 && t % h->K == 0) ckpt_copy(h, t / h->K, true);
            enqueue_step(h, t);
        }
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
    h->tape_ready = h->K > 0;
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
    h->tape_ready = false;
    if (use_persist(h) && h->K == 0) {
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        enqueue_reset(h, T);
        CU(cudaEventRecord(e0, h->stream));
        TRY(enqueue_persist(h, 0, T, 1));
        CU(cudaEventRecord(e1, h->stream));
        CU(cudaGetLastError());
        CU(cudaStreamSynchronize(h->stream));
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (kernel_ms) { kernel_ms[0] = ms; kernel_ms[1] = 0; kernel_ms[2] = 0; }
        if (launches) { launches[0] = 1; launches[1] = 0; launches[2] = 0; }
        h->t = T;
        h->T = T;
        h->n_bins = sim_n_bins(T, h->opt.obs_every);
        h->reset_done = true;
        TRY(copy_outputs(h, out));
        return check_device_error(h);
    }
    std::vector<cudaEvent_t> ev((size_t)4 * T + 2);
    for (auto &e : ev) CU(cudaEventCreate(&e));
    enqueue_reset(h, T);
    for (int t = 0; t < T; ++t) {
        CU(cudaEventRecord(ev[4 * t + 0], h->stream));
        enqueue_a(h, t, 0);
        CU(cudaEventRecord(ev[4 * t + 1], h->stream));
        CU(cudaEventRecord(ev[4 * t + 2], h->stream));
        enqueue_b(h, t);
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

extern "C" int sim_backward(sim_handle h, const float *dL_dcounts, const float *dL_dxT,
                            int32_t inputs_on_device, sim_grads *out) {
    if (!h || !dL_dcounts || !out) return SIM_EINVAL;
    if (h->K <= 0) return fail(h, SIM_ESTATE, "sim_backward needs options.ckpt_every > 0");
    if (!h->tape_ready) return fail(h, SIM_ESTATE, "sim_backward needs a recorded sim_rollout just before");
    CU(cudaSetDevice(h->device));
    TRY(check_device_error(h));
    const int T = h->T, K = h->K, L = h->L, V = h->V, N = h->N, S = h->S, F = h->F;
    const int nb = h->n_bins, obs = h->opt.obs_every;
    const int nseg = (T + K - 1) / K;
    // adjoint of C_j at the end of each bin and its suffix sums (host, small)
    std::vector<float> yb((size_t)nb * L);
    CU(cudaMemcpyAsync(yb.data(), dL_dcounts, yb.size() * sizeof(float),
                       inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    std::vector<double> cb((size_t)nb * L), cs((size_t)(nb + 1) * L, 0.0);
    for (int bb = 0; bb < nb; ++bb)
        for (int j = 0; j < L; ++j)
            cb[(size_t)bb * L + j] = (double)yb[(size_t)bb * L + j] -
                                     (bb + 1 < nb ? (double)yb[(size_t)(bb + 1) * L + j] : 0.0);
    for (int bb = nb - 1; bb >= 0; --bb)
        for (int j = 0; j < L; ++j) cs[(size_t)bb * L + j] = cs[(size_t)(bb + 1) * L + j] + cb[(size_t)bb * L + j];
    if (h->device < 0 || h->device >= 64) return fail(h, SIM_EINVAL, "device index");
    // carve the workspace: one layout routine sizes it (from base 0) and then
    // hands out the sub-arrays (from the buffer)
    const int n_gw = (L + kGwLinks - 1) / kGwLinks;
    // recomputation beside the reverse pass, or before it in one persistent
    // recording launch per segment.  Two tape sets, by segment parity: the
    // Jacobian kernel of a segment reads its set while the next segment is
    // recorded into the other.
    const bool overlap = h->recompute != SIM_RECOMPUTE_SERIAL || !use_persist(h);
    BwdDev b = h->b;
    BwdDev bt[2] = {h->b, h->b};
    float2 *d_Cbar = nullptr, *d_Csuf = nullptr;
    double *d_gw_part = nullptr;
    float *d_dxT_w = nullptr, *d_gout = nullptr;
    auto carve = [&](uintptr_t base) -> size_t {
        uintptr_t wp = base;
        auto take = [&](size_t n, size_t sz) {
            void *p = (void *)wp;
            wp += (std::max<size_t>(n, 1) * sz + 255) & ~(size_t)255;
            return p;
        };
        for (int ts = 0; ts < 2; ++ts) {
            BwdDev &q = bt[ts];
            q.tpos = (float *)take((size_t)(K + 1) * S, sizeof(float));
            q.tvid = (int *)take(S, sizeof(int));
            q.tent = (int *)take((size_t)K * L, sizeof(int));
            q.tlq = (int4 *)take((size_t)(K + 1) * L, sizeof(int4));
            q.ttag = (int8_t *)take((size_t)K * S, 1);
            q.tcrec = (int4 *)take((size_t)K * L, sizeof(int4));
            q.tnrec = (int2 *)take((size_t)K * V, sizeof(int2));
            q.tW = (unsigned long long *)take((size_t)K * L, sizeof(unsigned long long));
            q.tmkey = (float *)take((size_t)K * (L + V), sizeof(float));
            q.Z = (double *)take((size_t)K * L, sizeof(double));
            q.SA = (double *)take((size_t)K * L, sizeof(double));
            q.ebuf = (float *)take((size_t)K * (L + V), sizeof(float));
            q.abuf = (float2 *)take((size_t)K * (L + V), sizeof(float2));
        }
        b.xbar = (float2 *)take(N, sizeof(float2));
        b.A = (float2 *)take(S, sizeof(float2));
        b.cursor = (int *)take(N, sizeof(int));
        b.rdup = (unsigned char *)take(N, 1);
        b.eadj = (float2 *)take((size_t)N * h->route_cap, sizeof(float2));
        b.gu = (double *)take(L, sizeof(double)); b.gs = (double *)take(L, sizeof(double));
        b.ga = (double *)take(L, sizeof(double)); b.gU = (double *)take(L, sizeof(double));
        b.gG = (double *)take(L, sizeof(double));
        b.gao = (double *)take(1, sizeof(double));
        b.glam = (double *)take(std::max(h->n_od, 1), sizeof(double));
        d_Cbar = (float2 *)take((size_t)nb * L, sizeof(float2));
        d_Csuf = (float2 *)take((size_t)(nb + 1) * L, sizeof(float2));
        d_dxT_w = (float *)take(N, sizeof(float));
        d_gout = (float *)take((size_t)5 * L + std::max(F, 1) + 1 + std::max(h->n_od, 1), sizeof(float));
        d_gw_part = (double *)take((size_t)n_gw * std::max(F, 1), sizeof(double));
        return (size_t)(wp - base);
    };
    const size_t need = carve(0);
    if (!h->jstream) {                   // the reverse pass's streams and events
        int lo = 0, hi = 0;
        CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CU(cudaStreamCreateWithPriority(&h->vstream, cudaStreamNonBlocking, hi));
        CU(cudaStreamCreateWithPriority(&h->jstream, cudaStreamNonBlocking, hi));
        CU(cudaStreamCreateWithPriority(&h->rstream, cudaStreamNonBlocking, lo));
        CU(cudaEventCreateWithFlags(&h->ev_z, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_g, cudaEventDisableTiming));
        for (cudaEvent_t *e : {&h->ev_r[0], &h->ev_r[1], &h->ev_b[0], &h->ev_b[1]})
            CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    BwdLease lease{&g_bwd_pool[h->device], bwd_take(h->device, need), {h->stream, h->vstream, h->jstream, h->rstream}};
    BwdWs &ws = *lease.w;
    if (need > ws.cap) {                 // grow (the previous user of this workspace has synchronised)
        if (ws.buf) cudaFreeAsync(ws.buf, h->stream);
        ws.buf = nullptr;
        ws.cap = 0;
        cudaError_t e = pool_alloc(&ws.buf, need, h->device, h->stream);
        if (e != cudaSuccess) { ws.buf = nullptr; return fail(h, SIM_ENOMEM, "reverse-pass workspace: " + std::string(cudaGetErrorString(e))); }
        ws.cap = need;
    }
    carve((uintptr_t)ws.buf);
    // bin adjoints as double-float pairs (hi = nearest float, lo = nearest float of the rest)
    std::vector<float2> cb2(cb.size()), cs2(cs.size());
    auto split = [](double v) { const float hi = (float)v; return make_float2(hi, (float)(v - (double)hi)); };
    for (size_t k = 0; k < cb.size(); ++k) cb2[k] = split(cb[k]);
    for (size_t k = 0; k < cs.size(); ++k) cs2[k] = split(cs[k]);
    CU(cudaMemcpyAsync(d_Cbar, cb2.data(), cb2.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d_Csuf, cs2.data(), cs2.size() * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
    b.Cbar = d_Cbar;
    b.Csuf = d_Csuf;
    const float *dxT = nullptr;
    if (dL_dxT) {
        CU(cudaMemcpyAsync(d_dxT_w, dL_dxT, (size_t)N * sizeof(float),
                           inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        dxT = d_dxT_w;
    }
    for (double *p : {b.gu, b.gs, b.ga, b.gU, b.gG}) CU(cudaMemsetAsync(p, 0, (size_t)L * sizeof(double), h->stream));
    CU(cudaMemsetAsync(b.gao, 0, sizeof(double), h->stream));
    CU(cudaMemsetAsync(b.glam, 0, (size_t)std::max(b.n_od, 1) * sizeof(double), h->stream));
    // eadj needs no clearing: entry r of a vehicle is undone (and its adjoint
    // written) at the step of that entry, before any earlier step reads it
    CU(cudaMemsetAsync(b.A, 0, (size_t)S * sizeof(float2), h->stream));
    const long long n_init = std::max((long long)N, 32LL * L);
    k_bwd_init<<<(unsigned)((n_init + 255) / 256), 256, 0, h->stream>>>(h->d, b, dxT);
    k_route_scan<<<(int)(((size_t)N * 32 + 255) / 256), 256, 0, h->stream>>>(h->d, N, b);
    for (int ts = 0; ts < 2; ++ts) {                     // merge sums of both tape sets start from zero
        CU(cudaMemsetAsync(bt[ts].Z, 0, (size_t)K * L * sizeof(double), h->stream));
        CU(cudaMemsetAsync(bt[ts].SA, 0, (size_t)K * L * sizeof(double), h->stream));
    }
    // recomputation: no route log, counters into a scratch array
    DevSim dr = h->d;
    dr.route_log = nullptr;
    dr.step_delta = h->d_dummy;
    const size_t smem_a = (size_t)h->stage_max * sizeof(float);

    const int gS = (std::max(S, L) + 255) / 256;
    // Segments from the last.  The tape has two sets, by segment parity.  In
    // overlapped mode the recomputation of segment s - 1 (on the third stream,
    // two-kernel executor, whose blocks share SMs with the reverse kernels)
    // runs beside the reverse pass of segment s, which reads only its tape set
    // and static data.  A set is rewritten only after the Jacobian kernel that
    // read it last (ev_b); a reverse pass starts only once its set is recorded
    // (ev_r).
    auto with_set = [&](int ts) {
        BwdDev q = b;
        q.tpos = bt[ts].tpos; q.tvid = bt[ts].tvid; q.tent = bt[ts].tent; q.tlq = bt[ts].tlq; q.ttag = bt[ts].ttag;
        q.tcrec = bt[ts].tcrec; q.tnrec = bt[ts].tnrec; q.tW = bt[ts].tW; q.tmkey = bt[ts].tmkey;
        q.Z = bt[ts].Z; q.SA = bt[ts].SA; q.ebuf = bt[ts].ebuf; q.abuf = bt[ts].abuf;
        return q;
    };
    auto recompute = [&](int sg) -> int {
        const int t0 = sg * K, t1 = std::min(T, t0 + K), ts = sg & 1;
        const cudaStream_t rs = h->rstream;
        const BwdDev q = with_set(ts);
        CU(cudaStreamWaitEvent(rs, h->ev_b[ts], 0));
        ckpt_copy(h, sg, false, rs);
        CU(cudaMemsetAsync((t0 & 1) ? h->d.W1 : h->d.W0, 0, (size_t)L * sizeof(unsigned long long), rs));
        DevSim dq = dr;
        dq.tape_ent = q.tent;
        dq.tape_lq0 = q.tlq;
        dq.tape_K = K;
        for (int t = t0; t < t1; ++t) {            // each step writes its own tape record
            const size_t r = (size_t)(t - t0);
            dq.tag_tape = q.ttag + r * S;
            dq.tape_pos = q.tpos + r * S;
            dq.tape_vid = r == 0 ? q.tvid : nullptr;
            dq.tape_lq = q.tlq + r * L;
            dq.tape_crec = q.tcrec + r * L;
            dq.tape_nrec = q.tnrec + r * V;
            dq.tape_W = q.tW + r * L;
            dq.tape_mkey = q.tmkey + r * (L + V);
            k_step_a_tape<<<dq.nblk, kBlockA, smem_a, rs>>>(dq, t);
            k_step_b<<<(L + V + 255) / 256, 256, 0, rs>>>(dq, t);
        }
        dq.tape_W = nullptr;
        k_tape_pre<<<gS, 256, 0, rs>>>(dq, q, t1 - t0, t1 & 1);        // state at the end of the segment
        CU(cudaEventRecord(h->ev_r[ts], rs));
        return SIM_OK;
    };
    // the initial adjoints are read before any recomputation changes the state
    CU(cudaEventRecord(h->ev_b[0], h->stream));
    CU(cudaEventRecord(h->ev_b[1], h->stream));
    CU(cudaEventRecord(h->ev_g, h->stream));
    const cudaStream_t vs = h->vstream;                   // the reverse chain, high priority
    const int nlb = (L + kCfLinks - 1) / kCfLinks, npb = (V + nlb - 1) / nlb;
    CU(cudaStreamWaitEvent(vs, h->ev_g, 0));
    // one recording launch of the persistent executor for segment sg, on the
    // reverse chain's stream (serial mode)
    auto recompute_serial = [&](int sg) -> int {
        const int t0 = sg * K, t1 = std::min(T, t0 + K), ts = sg & 1;
        const BwdDev q = with_set(ts);
        CU(cudaStreamWaitEvent(vs, h->ev_b[ts], 0));
        CU(cudaMemsetAsync((t0 & 1) ? h->d.W1 : h->d.W0, 0, (size_t)L * sizeof(unsigned long long), vs));
        // the recording starts from the segment's checkpoint in place, and leaves
        // its end state there (no restore copy; no later step reads that checkpoint)
        DevSim dq = dr;
        dq.lq = h->ck.lq + (size_t)sg * L; dq.lstat = h->ck.lstat + (size_t)sg * L;
        dq.vac = h->ck.vac + (size_t)sg * L; dq.lpos = h->ck.lpos + (size_t)sg * L;
        dq.sentry = h->ck.sentry + (size_t)sg * S; dq.saux = h->ck.saux + (size_t)sg * S;
        dq.pos0 = dq.pos1 = h->ck.pos + (size_t)sg * S;
        dq.fifo_ptr = h->ck.fifo + (size_t)sg * V; dq.vstate = h->ck.vstate + (size_t)sg * N;
        dq.tag_tape = q.ttag; dq.tape_pos = q.tpos; dq.tape_vid = q.tvid; dq.tape_lq = q.tlq;
        dq.tape_ent = q.tent; dq.tape_lq0 = q.tlq; dq.tape_K = K; dq.tape_mkey = q.tmkey;
        dq.tape_crec = q.tcrec; dq.tape_nrec = q.tnrec; dq.tape_W = q.tW;
        TRY(enqueue_persist_d(h, dq, t0, t1, 0, true, vs));
        dq.tape_W = nullptr;
        k_tape_pre<<<gS, 256, 0, vs>>>(dq, q, t1 - t0, t1 & 1);
        return SIM_OK;
    };
    if (overlap) TRY(recompute(nseg - 1));
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int t0 = sg * K, t1 = std::min(T, t0 + K), ts = sg & 1;
        if (overlap) {
            if (sg > 0) TRY(recompute(sg - 1));
            CU(cudaStreamWaitEvent(vs, h->ev_r[ts], 0));
        } else {
            TRY(recompute_serial(sg));
        }
        const BwdDev q = with_set(ts);
        // Per step on the chain's stream: the merge adjoint and car-following in
        // one launch.  The merge sums start from zero: zeroed at the start, and
        // after each Jacobian kernel that read them (before ev_b).
        // A step that follows the previous one directly is launched as its
        // programmatic dependent: it issues its tape loads while that one ends.
        for (int t = t1 - 1; t >= t0; --t) {
            const int rec = t - t0;
            const bool at_obs = (t + 1) % obs == 0 || t + 1 == T;
            if (at_obs) k_bwd_obs<<<(L * 32 + 255) / 256, 256, 0, vs>>>(dr, q, rec + 1, t / obs);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(nlb);
            cfg.blockDim = dim3(kBwdThreads);
            cfg.stream = vs;
            cudaLaunchAttribute pdl[1];
            pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            pdl[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = pdl;
            cfg.numAttrs = (t + 1 < t1 && !at_obs) ? 1 : 0;
            CU(cudaLaunchKernelEx(&cfg, k_bwd_step, dr, q, rec, t, t / obs, npb));
        }
        // the segment's Jacobians on the second stream, beside the next segment
        CU(cudaEventRecord(h->ev_z, vs));
        CU(cudaStreamWaitEvent(h->jstream, h->ev_z, 0));
        const long long ng = (long long)(t1 - t0) * (L + V);
        k_bwd_node_g<<<(unsigned)((ng + 255) / 256), 256, 0, h->jstream>>>(dr, q, t0, t1 - t0);
        CU(cudaMemsetAsync(q.Z, 0, (size_t)K * L * sizeof(double), h->jstream));
        CU(cudaMemsetAsync(q.SA, 0, (size_t)K * L * sizeof(double), h->jstream));
        CU(cudaEventRecord(h->ev_b[ts], h->jstream));      // this tape set may be rewritten
        CU(cudaGetLastError());
    }
    CU(cudaEventRecord(h->ev_z, vs));
    CU(cudaStreamWaitEvent(h->stream, h->ev_z, 0));       // the handle's stream resumes after the chain
    CU(cudaEventRecord(h->ev_g, h->jstream));
    CU(cudaStreamWaitEvent(h->stream, h->ev_g, 0));       // and after the last Jacobian kernel
    // parameter gradients
    float *go = d_gout;
    float *gu = go, *gk = go + L, *ga = go + 2 * L, *gbeta = go + 3 * L, *gc = go + 4 * L, *gw = go + 5 * L;
    float *gao = gw + std::max(F, 1), *gl = gao + 1;
    const int nfin = std::max(std::max(L, F), std::max(b.n_od, 1));
    if (F > 0) k_bwd_gw_part<<<n_gw, kGwLinks, 0, h->stream>>>(h->d, b, h->d_phi, h->d_psi, d_gw_part);
    k_bwd_finalize<<<(nfin + 255) / 256, 256, 0, h->stream>>>(h->d, b, h->d_kappa, h->d_beta, h->d_cost, d_gw_part,
                                                               n_gw, h->opt.dn, gu, gk, ga, gbeta, gc, gw, gao, gl);
    CU(cudaGetLastError());
    const cudaMemcpyKind kd = out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const std::pair<float *, const float *> outs[] = {
        {out->d_u, gu}, {out->d_kappa, gk}, {out->d_alpha, ga}, {out->d_beta, gbeta}, {out->d_cost, gc}};
    for (auto &o : outs)
        if (o.first) CU(cudaMemcpyAsync(o.first, o.second, (size_t)L * sizeof(float), kd, h->stream));
    if (out->d_w && F) CU(cudaMemcpyAsync(out->d_w, gw, (size_t)F * sizeof(float), kd, h->stream));
    if (out->d_alpha_origin) CU(cudaMemcpyAsync(out->d_alpha_origin, gao, sizeof(float), kd, h->stream));
    if (out->d_od_lambda && b.n_od) CU(cudaMemcpyAsync(out->d_od_lambda, gl, (size_t)b.n_od * sizeof(float), kd, h->stream));
    // the recomputation left the state of an earlier time: a new run must reset
    h->tape_ready = false;
    h->reset_done = false;
    CU(cudaStreamSynchronize(h->stream));
    return check_device_error(h);
}

extern "C" int sim_get_state(sim_handle h, sim_state_view *out) {
    if (!h || !out) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    const int L = h->L, N = h->N, V = h->V, S = h->S;
    std::vector<int4> lq(L);
    std::vector<float> pos(S);
    std::vector<int2> saux(S);
    std::vector<int> sentry(S), vstate(N), fptr(V);
    CU(cudaMemcpyAsync(lq.data(), h->d.lq, L * sizeof(int4), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(pos.data(), (h->t & 1) ? h->d.pos1 : h->d.pos0, S * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(saux.data(), h->d.saux, S * sizeof(int2), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(sentry.data(), h->d.sentry, S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(vstate.data(), h->d.vstate, N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(fptr.data(), h->d.fifo_ptr, V * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < N; ++i) {
        const int s = vstate[i] >= 0 ? -1 : vstate[i];
        if (out->veh_link) out->veh_link[i] = s;
        if (out->veh_pos) out->veh_pos[i] = 0.0;
        if (out->veh_rank) out->veh_rank[i] = -1;
        if (out->veh_entry) out->veh_entry[i] = -1;
    }
    for (int j = 0; j < L; ++j) {
        const int base = h->lst_host[4 * j], cap = h->lst_host[4 * j + 1];
        for (int k = 0; k < lq[j].y; ++k) {
            int idx = lq[j].x + k;
            if (idx >= cap) idx -= cap;
            const int v = saux[base + idx].x;
            if (v < 0 || v >= N) return fail(h, SIM_ESTATE, "corrupt queue");
            if (out->veh_link) out->veh_link[v] = j;
            if (out->veh_pos) out->veh_pos[v] = pos[base + idx];
            if (out->veh_rank) out->veh_rank[v] = k;
            if (out->veh_entry) out->veh_entry[v] = sentry[base + idx];
        }
        if (out->link_credit) out->link_credit[j] = lq[j].z;
        if (out->link_exits) out->link_exits[j] = lq[j].w;
    }
    if (out->fifo_off)
        for (int n = 0; n < V; ++n) out->fifo_off[n] = fptr[n] - h->fifo_beg[n];
    return SIM_OK;
}

extern "C" int sim_set_state(sim_handle h, const sim_state_view *in, int32_t t) {
    if (!h || !in) return SIM_EINVAL;
    if (!h->reset_done) return fail(h, SIM_ESTATE, "sim_reset first");
    if (t < 0 || t > h->T) return fail(h, SIM_ESTATE, "step outside the horizon");
    if (!in->veh_link || !in->veh_pos || !in->veh_rank || !in->veh_entry || !in->link_credit || !in->link_exits ||
        !in->fifo_off)
        return fail(h, SIM_EINVAL, "every field of the state is required");
    CU(cudaSetDevice(h->device));
    const int L = h->L, N = h->N, V = h->V, S = h->S;
    std::vector<int4> lq(L);
    std::vector<float> pos(S, 0.0f);
    std::vector<int2> saux(S, make_int2(-1, -1));
    std::vector<int> sentry(S, 0), vstate(N), fptr(V), cnt(L, 0);
    std::vector<int4> lstat(L);
    std::vector<longlong2> lpos(L);
    std::vector<int> dz(N);
    CU(cudaMemcpyAsync(dz.data(), h->d.dest_zone, (size_t)N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    long long waiting = 0, queued = 0;
    for (int n = 0; n < V; ++n) {
        const int len = h->fifo_beg[n + 1] - h->fifo_beg[n];
        if (in->fifo_off[n] < 0 || in->fifo_off[n] > len) return fail(h, SIM_EINVAL, "origin queue offset out of range");
        fptr[n] = h->fifo_beg[n] + in->fifo_off[n];
        queued += len - in->fifo_off[n];
    }
    for (int i = 0; i < N; ++i) {
        const int j = in->veh_link[i];
        if (j < kVehArrived || j >= L) return fail(h, SIM_EINVAL, "vehicle link out of range");
        vstate[i] = j;
        if (j == kVehWaiting) { ++waiting; continue; }
        if (j < 0) continue;
        const int cap = h->lst_host[4 * j + 1], k = in->veh_rank[i];
        const double x = in->veh_pos[i];
        if (k < 0 || k >= cap - 1) return fail(h, SIM_EINVAL, "rank out of range");
        if (!(x >= 0.0 && x <= (double)h->length[j])) return fail(h, SIM_EINVAL, "position outside its link");
        const int slot = h->lst_host[4 * j] + k;
        if (saux[slot].x >= 0) return fail(h, SIM_EINVAL, "two vehicles with the same rank");
        saux[slot] = make_int2(i, dz[i]);
        pos[slot] = (float)x;
        sentry[slot] = in->veh_entry[i];
        cnt[j] += 1;
    }
    if (waiting != queued) return fail(h, SIM_EINVAL, "waiting vehicles do not match the origin queues");
    for (int j = 0; j < L; ++j) {
        const int base = h->lst_host[4 * j];
        for (int k = 0; k < cnt[j]; ++k)
            if (saux[base + k].x < 0) return fail(h, SIM_EINVAL, "ranks of a link are not 0..n-1");
        if (in->link_credit[j] < 0 || in->link_credit[j] > h->lst_host[4 * j + 3])
            return fail(h, SIM_EINVAL, "credit out of range");
        lq[j] = make_int4(0, cnt[j], (int)in->link_credit[j], (int)in->link_exits[j]);
        // the open bin restarts at t: C at its start, position sum at t
        long long past = 0, psum = 0;
        for (int k = 0; k < cnt[j]; ++k) {
            const float x = pos[base + k];
            past += x >= h->length[j] * 0.5f;
            psum += llrintf(x * 65536.0f);
        }
        lstat[j] = make_int4(0, 0, 0, (int)(in->link_exits[j] + past));
        lpos[j] = make_longlong2(psum, 0);
    }
    DevSim &d = h->d;
    float *pc = (t & 1) ? d.pos1 : d.pos0;
    CU(cudaMemcpyAsync(d.lq, lq.data(), L * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(pc, pos.data(), (size_t)S * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.saux, saux.data(), (size_t)S * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.sentry, sentry.data(), (size_t)S * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.vstate, vstate.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.fifo_ptr, fptr.data(), (size_t)V * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.lstat, lstat.data(), L * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.lpos, lpos.data(), L * sizeof(longlong2), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemsetAsync(d.W0, 0, L * sizeof(unsigned long long), h->stream));
    CU(cudaMemsetAsync(d.W1, 0, L * sizeof(unsigned long long), h->stream));
    const std::vector<int4> crec(L, make_int4(-1, kTgtNone, 0, 0));
    const std::vector<int2> nrec(V, make_int2(-1, kTgtNone));
    CU(cudaMemcpyAsync(d.crec, crec.data(), L * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(d.nrec, nrec.data(), V * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    k_set_flags<<<(L + 255) / 256, 256, 0, h->stream>>>(d, t);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
    h->t = t;
    h->tape_ready = false;
    return SIM_OK;
}

extern "C" int sim_get_records(sim_handle h, sim_records *out) {
    if (!h || !out) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    const int L = h->L, V = h->V;
    std::vector<int4> lc(L);
    std::vector<int2> nc(V);
    std::vector<unsigned long long> W(L);
    const int p = (h->t - 1) & 1;
    CU(cudaMemcpyAsync(lc.data(), h->d.crec, L * sizeof(int4), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(nc.data(), h->d.nrec, V * sizeof(int2), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(W.data(), p ? h->d.W1 : h->d.W0, L * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < L; ++j) {
        if (out->link_cand) out->link_cand[j] = lc[j].y == kTgtNone ? -1 : lc[j].x;
        if (out->link_target) out->link_target[j] = lc[j].y;
        if (out->link_in) out->link_in[j] = W[j] ? (int)(~(uint32_t)(W[j] & 0xffffffffull)) : -1;
    }
    for (int n = 0; n < V; ++n) {
        if (out->node_cand) out->node_cand[n] = nc[n].y == kTgtNone ? -1 : nc[n].x;
        if (out->node_target) out->node_target[n] = nc[n].y;
    }
    return SIM_OK;
}

extern "C" int sim_set_stream(sim_handle h, void *stream) {
    if (!h) return SIM_EINVAL;
    CU(cudaSetDevice(h->device));
    CU(cudaStreamSynchronize(h->stream));
    if (stream) {
        if (h->own_stream) CU(cudaStreamDestroy(h->stream));
        h->own_stream = false;
        h->stream = (cudaStream_t)stream;
    }
    return SIM_OK;
}

/* queue slots staged in shared memory per link block of k_step_a */
extern "C" int sim_set_stage(sim_handle h, int32_t slots) {
    if (!h) return SIM_EINVAL;
    if (slots < 256 || slots > 8192) return fail(h, SIM_EINVAL, "stage must be in [256, 8192] slots");
    if (slots != h->stage) {
        h->stage = slots;
        TRY(build_blocks(h));
        for (auto &g : h->graphs) cudaGraphExecDestroy(g.second);
        h->graphs.clear();
    }
    return SIM_OK;
}

extern "C" int sim_set_executor(sim_handle h, int32_t executor) {
    if (!h) return SIM_EINVAL;
    if (executor != SIM_EXEC_AUTO && executor != SIM_EXEC_STEP && executor != SIM_EXEC_PERSISTENT)
        return fail(h, SIM_EINVAL, "unknown executor");
    if (executor == SIM_EXEC_PERSISTENT && !h->persist_ok)
        return fail(h, SIM_EINVAL, "persistent executor unavailable: " + h->persist_why);
    h->executor = executor;
    return SIM_OK;
}

extern "C" int sim_set_partition_weights(sim_handle h, const float *w) {
    if (!h) return SIM_EINVAL;
    std::vector<long long> pw;
    if (w) {
        double m = 0.0;
        for (int j = 0; j < h->L; ++j) {
            if (!std::isfinite(w[j]) || w[j] < 0.0f) return fail(h, SIM_EINVAL, "partition weights must be finite and >= 0");
            m = std::max(m, (double)w[j]);
        }
        if (!(m > 0.0)) return fail(h, SIM_EINVAL, "partition weights are all zero");
        pw.resize(h->L);
        for (int j = 0; j < h->L; ++j) pw[j] = 1 + std::llround((double)w[j] / m * (double)(1 << 20));
    }
    CU(cudaSetDevice(h->device));
    CU(cudaStreamSynchronize(h->stream));       // launches in flight read the old bounds
    const bool was_ok = h->persist_ok;
    h->pw.swap(pw);
    const int rc = build_groups(h);
    if (rc == SIM_OK && (h->persist_ok || !was_ok)) return SIM_OK;
    const std::string why = h->persist_why;
    h->pw.swap(pw);                             // back to the previous weights
    TRY(build_groups(h));
    return rc ? rc : fail(h, SIM_EINVAL, "no persistent grouping with these weights: " + why);
}

extern "C" int32_t sim_persist_groups(sim_handle h, int32_t *first_link) {
    if (!h) return -1;
    if (!h->persist_ok) return 0;
    if (first_link) {
        if (cudaSetDevice(h->device) != cudaSuccess) return -1;
        if (cudaMemcpy(first_link, h->d_grp, (size_t)(h->G + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    }
    return h->G;
}

extern "C" int sim_test_barrier_timeout(sim_handle h, int32_t missing) {
    if (!h || missing < 0) return SIM_EINVAL;
    if (!h->persist_ok) return fail(h, SIM_EINVAL, "persistent executor unavailable: " + h->persist_why);
    h->bar_extra = missing;
    return SIM_OK;
}

extern "C" int sim_set_recompute(sim_handle h, int32_t mode) {
    if (!h) return SIM_EINVAL;
    if (mode != SIM_RECOMPUTE_OVERLAP && mode != SIM_RECOMPUTE_SERIAL) return fail(h, SIM_EINVAL, "unknown recompute mode");
    h->recompute = mode;
    return SIM_OK;
}

extern "C" int32_t sim_get_executor(sim_handle h) {
    if (!h) return -1;
    return use_persist(h) ? SIM_EXEC_PERSISTENT : SIM_EXEC_STEP;
}

extern "C" int32_t sim_time(sim_handle h) { return h ? h->t : -1; }
extern "C" void *sim_get_stream(sim_handle h) { return h ? (void *)h->stream : nullptr; }
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

// ============================================================================
// Batches: many handles advanced by one launch per phase and step
// ============================================================================

struct sim_batch_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<sim_ctx *> m;
    std::vector<cudaStream_t> saved_streams;
    DevSim *d_ds = nullptr;
    int2 *d_bmapA = nullptr, *d_bmapB = nullptr;
    int *d_t = nullptr, *d_T = nullptr, *d_mode = nullptr;
    CkDev *d_ck = nullptr;
    int nA = 0, nB = 0, maxS = 0;
    size_t smem = 0;
    bool any_tape = false;
    std::vector<int> hT, hmode;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<void *> allocs;
    std::string err;
    // persistent batch executor (one cooperative launch per advance)
    int executor = SIM_EXEC_AUTO;
    bool bp_ok = false;
    std::string bp_why;
    int bp_grid = 0;
    size_t bp_smem = 0;
    int2 *d_itA = nullptr, *d_itB = nullptr;
    int nIA = 0, nIB = 0;
    unsigned *d_bar = nullptr;
    int *d_berr = nullptr;
    unsigned char *d_ckstep = nullptr;
    int ckstep_cap = 0;
    int bar_extra = 0;                   // test hook: missing arrivals at the next launch's barriers
};

static int bfail(sim_batch_ctx *b, int code, const std::string &msg) {
    if (b) b->err = msg; else g_create_err = msg;
    return code;
}

#define BCU(call)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return bfail(b, SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static int balloc(sim_batch_ctx *b, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = pool_alloc(&q, std::max<size_t>(n, 1) * sizeof(T), b->device, b->stream);
    if (e != cudaSuccess) return bfail(b, SIM_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    b->allocs.push_back(q);
    *p = (T *)q;
    return SIM_OK;
}

static int batch_upload_member(sim_batch_ctx *b, int k) {
    sim_ctx *h = b->m[k];
    BCU(cudaMemcpyAsync(b->d_ds + k, &h->d, sizeof(DevSim), cudaMemcpyHostToDevice, b->stream));
    CkDev c{};
    if (h->K > 0) {
        c.K = h->K; c.L = h->L; c.S = h->S; c.V = h->V; c.N = h->N;
        c.lq = h->ck.lq; c.lstat = h->ck.lstat; c.vac = h->ck.vac; c.sentry = h->ck.sentry; c.fifo = h->ck.fifo;
        c.vstate = h->ck.vstate; c.pos = h->ck.pos; c.saux = h->ck.saux; c.lpos = h->ck.lpos;
    }
    BCU(cudaMemcpyAsync(b->d_ck + k, &c, sizeof(CkDev), cudaMemcpyHostToDevice, b->stream));
    return SIM_OK;
}

static void batch_release(sim_batch_ctx *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    for (void *p : b->allocs) cudaFreeAsync(p, b->stream);
    b->allocs.clear();
    if (b->d_ckstep) cudaFreeAsync(b->d_ckstep, b->stream);
    b->d_ckstep = nullptr;
    b->ckstep_cap = 0;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (size_t k = 0; k < b->m.size() && k < b->saved_streams.size(); ++k) b->m[k]->stream = b->saved_streams[k];
}

static size_t g_attr_bp[64];

// Work items of the persistent batch executor: 32 links, 32 origin nodes or 32
// transfer elements of one member each.  The executor is left off (with the
// reason) when the device cannot run the cooperative launch.
static int batch_persist_setup(sim_batch_ctx *b) {
    const int n = (int)b->m.size();
    std::vector<int2> iA, iB;
    for (int k = 0; k < n; ++k) {
        const sim_ctx *h = b->m[k];
        for (int j0 = 0; j0 < h->L; j0 += 32) iA.push_back(make_int2(k, j0));
        for (int n0 = 0; n0 < h->V; n0 += 32) iA.push_back(make_int2(k, n0 | kItemNode));
        for (int i0 = 0; i0 < h->L + h->V; i0 += 32) iB.push_back(make_int2(k, i0));
    }
    b->nIA = (int)iA.size();
    b->nIB = (int)iB.size();
    int rc;
    if ((rc = balloc(b, &b->d_itA, iA.size())) || (rc = balloc(b, &b->d_itB, iB.size())) ||
        (rc = balloc(b, &b->d_bar, 1)))
        return rc;
    BCU(cudaMemcpyAsync(b->d_itA, iA.data(), iA.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_itB, iB.data(), iB.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    b->bp_ok = false;
    if (n > kBMaxMembers) { b->bp_why = "more members than one launch holds"; return SIM_OK; }
    int coop = 0, nsm = 0, occ = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (!coop) { b->bp_why = "no cooperative launch on this device"; return SIM_OK; }
    b->bp_smem = b_dyn_bytes(n);
    if (raise_smem_attr(k_batch_persist, g_attr_bp, b->device, b->bp_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_persist, kBT, b->bp_smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        b->bp_why = "the persistent batch kernel does not fit on an SM";
        return SIM_OK;
    }
    b->bp_grid = nsm;
    b->bp_ok = true;
    return SIM_OK;
}

static bool batch_use_persist(const sim_batch_ctx *b) { return b->bp_ok && b->executor != SIM_EXEC_STEP; }

// A lone running member advances on its own persistent executor (queues in
// shared memory), which is faster for one member than the warp-item batch
// kernel.  Both leave the state in the same format at a launch boundary, so
// the executors can alternate between advances.  Returns -1 when the batch has
// not exactly one running member (or it has no persistent executor).
static int batch_solo_member(const sim_batch_ctx *b) {
    int k1 = -1;
    for (int k = 0; k < (int)b->m.size(); ++k) {
        if (b->hmode[k] == kModeDone) continue;
        if (k1 >= 0) return -1;
        k1 = k;
    }
    return (k1 >= 0 && use_persist(b->m[k1])) ? k1 : -1;
}

static int batch_advance_solo(sim_batch_ctx *b, int k, int n_steps) {
    sim_ctx *h = b->m[k];
    const int T = b->hT[k];
    int t = h->t, mode = b->hmode[k], left = n_steps;
    if (mode == kModeRun) {
        const int t_end = std::min(T, t + left);
        while (t < t_end) {                      // segments between checkpoints
            int t1 = t_end;
            if (h->K > 0) {
                if (t % h->K == 0) ckpt_copy(h, t / h->K, true);
                t1 = std::min(t_end, (t / h->K + 1) * h->K);
            }
            const bool fin = t1 == T && left > t1 - h->t;
            if (enqueue_persist(h, t, t1, fin ? 1 : 0)) return bfail(b, SIM_ECUDA, h->err);
            t = t1;
        }
        left -= t - h->t;
        // at the horizon: the observation-only pass ran with the last segment
        // if a step was left for it, else it is the member's next step
        if (t == T) mode = left > 0 ? kModeDone : kModeFinal;
    } else if (mode == kModeFinal) {
        if (enqueue_persist(h, T, T, 1)) return bfail(b, SIM_ECUDA, h->err);
        mode = kModeDone;
    }
    BCU(cudaMemcpyAsync(b->d_t + k, &t, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_mode + k, &mode, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));       // the host values above are stack variables
    return SIM_OK;
}

// One cooperative launch advancing every running member by up to n_steps steps.
static int batch_launch_persist(sim_batch_ctx *b, int n_steps) {
    const int n = (int)b->m.size();
    std::vector<unsigned char> ck((size_t)n_steps, 0);
    if (b->any_tape) {
        for (int k = 0; k < n; ++k) {
            const sim_ctx *h = b->m[k];
            if (h->K <= 0 || b->hmode[k] != kModeRun) continue;
            for (int s = 0; s < n_steps && h->t + s < b->hT[k]; ++s)
                if ((h->t + s) % h->K == 0) ck[s] = 1;
        }
    }
    if (b->ckstep_cap < n_steps) {
        if (b->d_ckstep) cudaFreeAsync(b->d_ckstep, b->stream);
        b->d_ckstep = nullptr;
        b->ckstep_cap = 0;
        BCU(pool_alloc((void **)&b->d_ckstep, (size_t)n_steps, b->device, b->stream));
        b->ckstep_cap = n_steps;
    }
    BCU(cudaMemcpyAsync(b->d_ckstep, ck.data(), (size_t)n_steps, cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->stream));
    BCU(cudaMemsetAsync(b->d_berr, 0, sizeof(int), b->stream));
    BArgs a{};
    a.ds = b->d_ds;
    a.ck = b->d_ck;
    a.itA = b->d_itA;
    a.itB = b->d_itB;
    a.ckstep = b->d_ckstep;
    a.nA = b->nIA;
    a.nB = b->nIB;
    a.tvec = b->d_t;
    a.Tvec = b->d_T;
    a.mode = b->d_mode;
    a.n = n;
    a.n_steps = n_steps;
    a.bar = b->d_bar;
    a.berr = b->d_berr;
    a.bar_extra = b->bar_extra;
    b->bar_extra = 0;
    void *args[1] = {&a};
    BCU(cudaLaunchCooperativeKernel((const void *)k_batch_persist, dim3(b->bp_grid), dim3(kBT), args, b->bp_smem,
                                    b->stream));
    return SIM_OK;
}

extern "C" int sim_batch_create(const sim_handle *members, int32_t n, sim_batch *out) {
    if (!out) return bfail(nullptr, SIM_EINVAL, "null output");
    *out = nullptr;
    if (!members || n <= 0) return bfail(nullptr, SIM_EINVAL, "empty batch");
    sim_batch_ctx *b = new sim_batch_ctx();
    b->device = members[0]->device;
    b->stream = members[0]->stream;
    std::vector<int2> bmA, bmB;
    for (int k = 0; k < n; ++k) {
        sim_ctx *h = members[k];
        if (!h || h->device != b->device) { delete b; return bfail(nullptr, SIM_EINVAL, "members must be distinct handles on one device"); }
        for (int q = 0; q < k; ++q) if (members[q] == h) { delete b; return bfail(nullptr, SIM_EINVAL, "a handle appears twice"); }
        b->m.push_back(h);
        b->saved_streams.push_back(h->stream);
        for (int x = 0; x < h->d.nblk; ++x) bmA.push_back(make_int2(k, x));
        const int nb = (h->L + h->V + 255) / 256;
        for (int x = 0; x < nb; ++x) bmB.push_back(make_int2(k, x));
        b->smem = std::max(b->smem, (size_t)h->stage_max * sizeof(float));
        b->any_tape = b->any_tape || h->K > 0;
        b->maxS = std::max(b->maxS, std::max(h->S, std::max(h->L, h->N)));
    }
    int rc = SIM_OK;
    auto fin = [&](int code) { batch_release(b); g_create_err = b->err; delete b; return code; };
    if (cudaSetDevice(b->device) != cudaSuccess) return fin(bfail(b, SIM_ECUDA, "cudaSetDevice"));
    // every member works on the batch's stream while batched
    cudaStreamSynchronize(b->stream);
    for (int k = 0; k < n; ++k) { cudaStreamSynchronize(b->m[k]->stream); b->m[k]->stream = b->stream; }
    b->nA = (int)bmA.size();
    b->nB = (int)bmB.size();
    if ((rc = balloc(b, &b->d_ds, n)) || (rc = balloc(b, &b->d_ck, n)) || (rc = balloc(b, &b->d_bmapA, b->nA)) ||
        (rc = balloc(b, &b->d_bmapB, b->nB)) || (rc = balloc(b, &b->d_t, 2 * (size_t)n + 1)) || (rc = balloc(b, &b->d_T, n)))
        return fin(rc);
    // steps, modes and the barrier-timeout flag side by side: one read-back per advance
    b->d_mode = b->d_t + n;
    b->d_berr = b->d_t + 2 * n;
    if (cudaMemsetAsync(b->d_berr, 0, sizeof(int), b->stream) != cudaSuccess)
        return fin(bfail(b, SIM_ECUDA, "batch set-up"));
    // members already running in an earlier batch continue where they are
    std::vector<int> ht(n);
    b->hT.assign(n, 0);
    b->hmode.assign(n, kModeDone);
    for (int k = 0; k < n; ++k) {
        sim_ctx *h = b->m[k];
        b->hmode[k] = h->bmode;
        b->hT[k] = h->bmode == kModeDone ? 0 : h->T;
        ht[k] = h->bmode == kModeDone ? 0 : h->t;
    }
    if (cudaMemcpyAsync(b->d_bmapA, bmA.data(), bmA.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) ||
        cudaMemcpyAsync(b->d_bmapB, bmB.data(), bmB.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) ||
        cudaMemcpyAsync(b->d_t, ht.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream) ||
        cudaMemcpyAsync(b->d_T, b->hT.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream) ||
        cudaMemcpyAsync(b->d_mode, b->hmode.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream))
        return fin(bfail(b, SIM_ECUDA, "batch set-up copies"));
    for (int k = 0; k < n; ++k)
        if ((rc = batch_upload_member(b, k))) return fin(rc);
    if (raise_smem_attr(k_batch_a, g_attr_ba, b->device, b->smem) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fin(bfail(b, SIM_ECUDA, "batch set-up"));
    if ((rc = batch_persist_setup(b))) return fin(rc);
    *out = b;
    return SIM_OK;
}

extern "C" int sim_batch_start(sim_batch b, int32_t k, int32_t T) {
    if (!b || k < 0 || k >= (int)b->m.size()) return SIM_EINVAL;
    if (T < 1) return bfail(b, SIM_EINVAL, "horizon must be >= 1");
    sim_ctx *h = b->m[k];
    BCU(cudaSetDevice(b->device));
    int rc = ensure_T(h, T);
    if (rc) return bfail(b, rc, h->err);
    enqueue_reset(h, T);
    BCU(cudaGetLastError());
    if ((rc = batch_upload_member(b, k))) return rc;
    const int zero = 0, run = kModeRun;
    BCU(cudaMemcpyAsync(b->d_t + k, &zero, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_T + k, &T, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_mode + k, &run, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    b->hT[k] = T;
    b->hmode[k] = kModeRun;
    h->bmode = kModeRun;
    h->t = 0;
    h->T = T;
    h->n_bins = sim_n_bins(T, h->opt.obs_every);
    h->reset_done = false;           // reachable through the batch only until it finishes
    h->tape_ready = false;
    return SIM_OK;
}

static void batch_enqueue_steps(sim_batch_ctx *b, int n_steps) {
    const int n = (int)b->m.size();
    for (int s = 0; s < n_steps; ++s) {
        if (b->any_tape) k_batch_ckpt<<<dim3(64, n), 256, 0, b->stream>>>(b->d_ds, b->d_ck, b->d_t, b->d_mode);
        k_batch_a<<<b->nA, kBlockA, b->smem, b->stream>>>(b->d_ds, b->d_bmapA, b->d_t, b->d_mode);
        k_batch_b<<<b->nB, 256, 0, b->stream>>>(b->d_ds, b->d_bmapB, b->d_t, b->d_mode);
        k_batch_tick<<<(n + 255) / 256, 256, 0, b->stream>>>(n, b->d_t, b->d_T, b->d_mode);
    }
}

extern "C" int sim_batch_advance(sim_batch b, int32_t n_steps, int32_t *finished) {
    if (!b || n_steps < 0) return SIM_EINVAL;
    BCU(cudaSetDevice(b->device));
    const int n = (int)b->m.size();
    if (n_steps > 0 && batch_use_persist(b)) {
        const int solo = batch_solo_member(b);
        const int rc = solo >= 0 ? batch_advance_solo(b, solo, n_steps) : batch_launch_persist(b, n_steps);
        if (rc) return rc;
        BCU(cudaGetLastError());
    } else if (n_steps > 0) {
        auto it = b->graphs.find(n_steps);
        if (it == b->graphs.end() && n_steps >= 8) {
            cudaGraph_t g;
            BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            batch_enqueue_steps(b, n_steps);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (ce != cudaSuccess) return bfail(b, SIM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            cudaGraphExec_t ge;
            ce = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return bfail(b, SIM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
            it = b->graphs.emplace(n_steps, ge).first;
        }
        if (it != b->graphs.end()) BCU(cudaGraphLaunch(it->second, b->stream));
        else batch_enqueue_steps(b, n_steps);
        BCU(cudaGetLastError());
    }
    std::vector<int> tm(2 * (size_t)n + 1);
    BCU(cudaMemcpyAsync(tm.data(), b->d_t, tm.size() * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    const int *tv = tm.data(), *mode = tm.data() + n;
    if (tm[2 * (size_t)n]) return bfail(b, SIM_ETIMEOUT, "persistent batch: a grid barrier timed out");
    std::vector<int> just_done;
    for (int k = 0; k < n; ++k) {
        sim_ctx *h = b->m[k];
        if (mode[k] == kModeDone && b->hmode[k] != kModeDone) {        // finished its horizon
            h->t = h->T;
            h->reset_done = true;
            h->tape_ready = h->K > 0;
            just_done.push_back(k);
        } else if (mode[k] != kModeDone) {
            h->t = tv[k];
        }
        b->hmode[k] = mode[k];
        h->bmode = mode[k];
        if (finished) finished[k] = mode[k] == kModeDone;
    }
    // device errors are sticky and a failing step skips its write, so a member's
    // flag is read once, when it finishes its horizon
    for (int k : just_done) {
        const int rc = check_device_error(b->m[k]);
        if (rc) return bfail(b, rc, b->m[k]->err);
    }
    return SIM_OK;
}

extern "C" int sim_batch_set_executor(sim_batch b, int32_t executor) {
    if (!b) return SIM_EINVAL;
    if (executor != SIM_EXEC_AUTO && executor != SIM_EXEC_STEP && executor != SIM_EXEC_PERSISTENT)
        return bfail(b, SIM_EINVAL, "unknown executor");
    if (executor == SIM_EXEC_PERSISTENT && !b->bp_ok)
        return bfail(b, SIM_EINVAL, "persistent batch executor unavailable: " + b->bp_why);
    b->executor = executor;
    return SIM_OK;
}

extern "C" int sim_batch_test_barrier_timeout(sim_batch b, int32_t missing) {
    if (!b || missing < 0) return SIM_EINVAL;
    if (!b->bp_ok) return bfail(b, SIM_EINVAL, "persistent batch executor unavailable: " + b->bp_why);
    b->bar_extra = missing;
    return SIM_OK;
}

extern "C" int32_t sim_batch_get_executor(sim_batch b) {
    if (!b) return -1;
    return batch_use_persist(b) ? SIM_EXEC_PERSISTENT : SIM_EXEC_STEP;
}

extern "C" int sim_batch_rollout(sim_batch b, int32_t T) {
    if (!b) return SIM_EINVAL;
    for (int k = 0; k < (int)b->m.size(); ++k) {
        const int rc = sim_batch_start(b, k, T);
        if (rc) return rc;
    }
    return sim_batch_advance(b, T + 1, nullptr);
}

extern "C" int sim_batch_destroy(sim_batch b) {
    if (!b) return SIM_OK;
    cudaSetDevice(b->device);
    batch_release(b);
    delete b;
    return SIM_OK;
}

extern "C" const char *sim_batch_last_error(sim_batch b) { return b ? b->err.c_str() : g_create_err.c_str(); }

// ============================================================================
// Allocation-free forward rollout.
//
// For callers that may not allocate device memory: plug-ins embedded in a host
// process whose memory manager owns every device allocation (and may refuse or
// account for any cudaMalloc made behind its back), and real-time loops, where
// cudaMalloc / cudaFree can block the host and synchronise the device.  All
// simulator state of the call lives in one file-scope device array of fixed
// size that every GPU loading this library holds until the process exits;
// host-side set-up uses fixed-size static host buffers, which one mutex guards
// (calls from several host threads run one after another, whatever their
// devices).  The paper has no counterpart of this.
// ============================================================================

namespace {

constexpr size_t kStaticBytes = (size_t)16 << 20;      // device scratch: 16 MiB
constexpr int kStaticMaxV = 4096, kStaticMaxL = 8192, kStaticMaxN = 65536;
constexpr int kStaticMaxChoice = 8 * kStaticMaxL;      // entries of all choice sets
constexpr int kStaticMaxT = 8192;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// device address of g_static_scratch, looked up once per device
static void *g_static_addr[kStaticMaxDevices];

// host-side set-up buffers (no dynamic allocation), shared by every device and
// guarded by g_static_mutex from the first write to the last read
static std::mutex g_static_mutex;
static int hs_no_ptr[kStaticMaxV + 1], hs_no_idx[kStaticMaxL], hs_lo_idx[kStaticMaxChoice];
static int hs_lnode[4 * kStaticMaxL], hs_lst[4 * kStaticMaxL], hs_blk[kStaticMaxL + 1];
static int hs_fifo[kStaticMaxN], hs_fifo_beg[kStaticMaxV + 1], hs_fifo_dep[kStaticMaxN];
static int hs_fifo_aux[2 * kStaticMaxN], hs_fifo_end[kStaticMaxV], hs_fill[kStaticMaxV];
static int hs_counters[4 * kStaticMaxT];
static float hs_alpha[kStaticMaxL + 1];

struct Bump {           // carves 256-byte aligned sub-arrays out of the scratch
    unsigned char *base;
    size_t used;
    bool ok;
    template <class T>
    T *take(size_t n) {
        const size_t b = (std::max<size_t>(n, 1) * sizeof(T) + 255) & ~(size_t)255;
        if (used + b > kStaticBytes) { ok = false; return nullptr; }
        T *p = (T *)(base + used);
        used += b;
        return p;
    }
};

}  // namespace

extern "C" int sim_rollout_static(const sim_network *net, const sim_demand *dem, const sim_params *par,
                                  const sim_options *opt, int32_t T, sim_outputs *out) {
    if (!net || !dem || !par || !opt || !out) return SIM_EINVAL;
    const int V = net->V, L = net->L, N = dem->N, F = net->F, Z = net->Z;
    if (V <= 0 || L <= 0 || N < 0 || F < 0 || Z <= 0 || T < 1) return SIM_EINVAL;
    // every array the run reads must be given (the feature arrays only when F > 0,
    // the demand arrays only when N > 0)
    if (!net->tail || !net->head || !net->length || !net->q_fx || !net->node_zone || !net->dest_feat ||
        !par->u || !par->kappa || !par->alpha || !par->beta || !par->cost)
        return SIM_EINVAL;
    if (F > 0 && (!net->phi || !net->psi || !par->w)) return SIM_EINVAL;
    if (N > 0 && (!dem->origin || !dem->dest_zone || !dem->dep_step)) return SIM_EINVAL;
    // the step counters are summed on the host: device outputs cannot take them
    if (out->on_device && (out->n_waiting || out->n_on || out->n_arrived)) return SIM_EINVAL;
    if (V > kStaticMaxV || L > kStaticMaxL || N > kStaticMaxN || T > kStaticMaxT) return SIM_EOVERFLOW;
    if (!(opt->dt > 0) || !(opt->dn > 0) || opt->obs_every <= 0 || !(opt->tau_gumbel > 0)) return SIM_EINVAL;
    if (opt->device < 0 || opt->device >= kStaticMaxDevices) return SIM_EINVAL;
    for (int j = 0; j < L; ++j) {
        if (net->tail[j] < 0 || net->tail[j] >= V || net->head[j] < 0 || net->head[j] >= V) return SIM_EINVAL;
        if (!(net->length[j] > 0.0f) || net->q_fx[j] <= 0) return SIM_EINVAL;
        if (!(par->u[j] > 0.0f) || !(par->kappa[j] > 0.0f) || !(par->cost[j] > 0.0f)) return SIM_EINVAL;
        if (!((double)par->u[j] * opt->dt < 2000.0)) return SIM_EINVAL;
    }
    for (int n = 0; n < V; ++n)
        if (net->node_zone[n] < 0 || net->node_zone[n] >= Z) return SIM_EINVAL;
    for (int i = 0; i < N; ++i)
        if (dem->origin[i] < 0 || dem->origin[i] >= V || dem->dest_zone[i] < 0 || dem->dest_zone[i] >= Z ||
            dem->dep_step[i] < 0)
            return SIM_EINVAL;
    // ---- host set-up (same derived structures as sim_create) ----
    std::lock_guard<std::mutex> lock(g_static_mutex);
    for (int n = 0; n <= V; ++n) hs_no_ptr[n] = 0;
    for (int j = 0; j < L; ++j) hs_no_ptr[net->tail[j] + 1]++;
    for (int n = 0; n < V; ++n) hs_no_ptr[n + 1] += hs_no_ptr[n];
    for (int n = 0; n < V; ++n) hs_fill[n] = 0;
    for (int j = 0; j < L; ++j) hs_no_idx[hs_no_ptr[net->tail[j]] + hs_fill[net->tail[j]]++] = j;
    for (int n = 0; n < V; ++n) {
        const int deg = hs_no_ptr[n + 1] - hs_no_ptr[n];
        if (deg == 0 || deg > 32) return SIM_EINVAL;
    }
    int n_lo = 0;
    for (int l = 0; l < L; ++l) {
        const int n = net->head[l];
        int c = 0;
        for (int k = hs_no_ptr[n]; k < hs_no_ptr[n + 1]; ++k) c += net->head[hs_no_idx[k]] != net->tail[l];
        hs_lnode[4 * l + 0] = n;
        hs_lnode[4 * l + 1] = net->node_zone[n];
        hs_lnode[4 * l + 2] = n_lo;
        for (int k = hs_no_ptr[n]; k < hs_no_ptr[n + 1]; ++k) {
            const int m = hs_no_idx[k];
            if (!c || net->head[m] != net->tail[l]) {
                if (n_lo >= kStaticMaxChoice) return SIM_EOVERFLOW;
                hs_lo_idx[n_lo++] = m;
            }
        }
        hs_lnode[4 * l + 3] = n_lo;
    }
    const long long dn_fx = llrint((double)opt->dn * SIM_FX_ONE);
    long long S = 0;
    for (int j = 0; j < L; ++j) {
        const double cap = std::floor((double)net->length[j] * (double)par->kappa[j] / (double)opt->dn) + 2.0;
        if (cap > 1e6) return SIM_EOVERFLOW;
        hs_lst[4 * j + 0] = (int)S;
        hs_lst[4 * j + 1] = (int)cap;
        hs_lst[4 * j + 2] = net->q_fx[j];
        hs_lst[4 * j + 3] = (int)std::max<long long>(net->q_fx[j], dn_fx);
        S += (long long)cap;
    }
    if (S > (1ll << 24)) return SIM_EOVERFLOW;
    for (int i = 0; i < N; ++i) hs_fifo[i] = i;
    std::sort(hs_fifo, hs_fifo + N, [&](int a, int b) {
        if (dem->origin[a] != dem->origin[b]) return dem->origin[a] < dem->origin[b];
        if (dem->dep_step[a] != dem->dep_step[b]) return dem->dep_step[a] < dem->dep_step[b];
        return a < b;
    });
    for (int n = 0; n <= V; ++n) hs_fifo_beg[n] = 0;
    for (int i = 0; i < N; ++i) hs_fifo_beg[dem->origin[i] + 1]++;
    for (int n = 0; n < V; ++n) hs_fifo_beg[n + 1] += hs_fifo_beg[n];
    for (int n = 0; n < V; ++n) hs_fifo_end[n] = hs_fifo_beg[n + 1];
    for (int k = 0; k < N; ++k) {
        hs_fifo_dep[k] = dem->dep_step[hs_fifo[k]];
        hs_fifo_aux[2 * k] = hs_fifo[k];
        hs_fifo_aux[2 * k + 1] = dem->dest_zone[hs_fifo[k]];
    }
    const int stage = 4096;
    int nblk = 0, slots = 0, nl = 0, smax = 0;
    hs_blk[0] = 0;
    for (int j = 0; j < L; ++j) {
        const int cap = hs_lst[4 * j + 1];
        if (nl > 0 && (nl == kLinksPerBlock || slots + cap > stage)) {
            hs_blk[++nblk] = j;
            smax = std::max(smax, slots);
            slots = 0;
            nl = 0;
        }
        slots += cap;
        nl += 1;
    }
    hs_blk[++nblk] = L;
    smax = std::max(smax, slots);
    const int nblk_all = std::max(nblk, (V + kNodesPerBlock - 1) / kNodesPerBlock);
    if (nblk_all > kStaticMaxL) return SIM_EOVERFLOW;
    while (nblk < nblk_all) hs_blk[++nblk] = L;
    for (int j = 0; j < L; ++j) hs_alpha[j] = par->alpha[j];
    hs_alpha[L] = par->alpha_origin;
    // ---- device: carve the scratch (first call on a device looks up its address) ----
    if (cudaSetDevice(opt->device) != cudaSuccess) return SIM_ECUDA;
    if (!g_static_addr[opt->device]) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_static_scratch) != cudaSuccess || !a) return SIM_ECUDA;
        g_static_addr[opt->device] = a;
    }
    cudaStream_t s = (cudaStream_t)opt->stream;
    const int nb = sim_n_bins(T, opt->obs_every);
    Bump B{(unsigned char *)g_static_addr[opt->device], 0, true};
    DevSim d{};
    d.V = V; d.L = L; d.N = N; d.Z = Z; d.F = F;
    d.dn_fx = (int)dn_fx;
    d.obs_every = opt->obs_every;
    d.M = opt->M; d.eps_arr = opt->eps_arr; d.dt = opt->dt;
    d.key0 = (uint32_t)(opt->seed & 0xffffffffull);
    d.key1 = (uint32_t)(opt->seed >> 32) ^ opt->scenario_id;
    float4 *geo = B.take<float4>(L), *tinfo = B.take<float4>(L), *loinfo = B.take<float4>(n_lo),
           *noinfo = B.take<float4>(L);
    int4 *lst = B.take<int4>(L), *lnode = B.take<int4>(L);
    int *ebits = B.take<int>(L);
    float *alpha = B.take<float>(L + 1), *dest_feat = B.take<float>((size_t)Z * V);
    int *blk = B.take<int>(nblk + 1), *no_ptr = B.take<int>(V + 1), *node_zone = B.take<int>(V);
    int *fifo_end = B.take<int>(V), *fifo_dep = B.take<int>(N), *dest_zone = B.take<int>(N);
    int2 *fifo_list = B.take<int2>(N);
    float *len = B.take<float>(L), *u = B.take<float>(L), *kappa = B.take<float>(L), *beta = B.take<float>(L),
          *cost = B.take<float>(L), *phi = B.take<float>((size_t)L * F), *psi = B.take<float>((size_t)L * F),
          *w = B.take<float>(F);
    int *head = B.take<int>(L), *lo_idx = B.take<int>(n_lo), *no_idx = B.take<int>(L), *fifo_beg = B.take<int>(V);
    d.lq = B.take<int4>(L);
    d.crec = B.take<int4>(L);
    d.vac = B.take<int>(L);
    d.pos0 = B.take<float>(S);
    d.pos1 = B.take<float>(S);
    d.saux = B.take<int2>(S);
    d.sentry = B.take<int>(S);
    d.W0 = B.take<unsigned long long>(L);
    d.W1 = B.take<unsigned long long>(L);
    d.nrec = B.take<int2>(V);
    d.fifo_ptr = B.take<int>(V);
    d.vstate = B.take<int>(N);
    d.lstat = B.take<int4>(L);
    d.lpos = B.take<longlong2>(L);
    d.out_counts = B.take<int>((size_t)nb * L);
    d.out_speed = B.take<float>((size_t)nb * L);
    d.out_tt = B.take<float>((size_t)nb * L);
    d.step_delta = B.take<int>((size_t)4 * T);
    d.err = B.take<int>(4);
    if (!B.ok) return SIM_EOVERFLOW;
    d.geo = geo; d.ebits = ebits; d.tinfo = tinfo; d.loinfo = loinfo; d.noinfo = noinfo; d.lst = lst; d.lnode = lnode;
    d.alpha = alpha; d.dest_feat = dest_feat; d.blk_links = blk; d.nblk = nblk; d.no_ptr = no_ptr;
    d.npb = (V + nblk - 1) / nblk;
    d.node_zone = node_zone; d.fifo_end = fifo_end; d.fifo_dep = fifo_dep; d.dest_zone = dest_zone;
    d.fifo_list = fifo_list; d.tag_tape = nullptr;
#define SUP(dst, src, n) do { if ((n) > 0 && cudaMemcpyAsync((dst), (src), (size_t)(n) * sizeof(*(dst)), cudaMemcpyHostToDevice, s) != cudaSuccess) return SIM_ECUDA; } while (0)
    SUP(lst, (const int4 *)hs_lst, L);
    SUP(lnode, (const int4 *)hs_lnode, L);
    SUP(alpha, hs_alpha, L + 1);
    SUP(dest_feat, net->dest_feat, (size_t)Z * V);
    SUP(blk, hs_blk, nblk + 1);
    SUP(no_ptr, hs_no_ptr, V + 1);
    SUP(node_zone, net->node_zone, V);
    SUP(fifo_end, hs_fifo_end, V);
    SUP(fifo_dep, hs_fifo_dep, N);
    SUP(dest_zone, dem->dest_zone, N);
    SUP(fifo_list, (const int2 *)hs_fifo_aux, N);
    SUP(len, net->length, L);
    SUP(u, par->u, L);
    SUP(kappa, par->kappa, L);
    SUP(beta, par->beta, L);
    SUP(cost, par->cost, L);
    SUP(phi, net->phi, (size_t)L * F);
    SUP(psi, net->psi, (size_t)L * F);
    SUP(w, par->w, F);
    SUP(head, net->head, L);
    SUP(lo_idx, hs_lo_idx, n_lo);
    SUP(no_idx, hs_no_idx, L);
    SUP(fifo_beg, hs_fifo_beg, V);
#undef SUP
    // state that must start at zero: the whole run re-initialises it
    if (cudaMemsetAsync(d.pos0, 0, (size_t)S * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(d.pos1, 0, (size_t)S * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(d.saux, 0xff, (size_t)S * sizeof(int2), s) != cudaSuccess ||
        cudaMemsetAsync(d.sentry, 0, (size_t)S * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(d.step_delta, 0, (size_t)4 * T * sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(d.out_counts, 0, (size_t)nb * L * sizeof(int), s) != cudaSuccess)
        return SIM_ECUDA;
    k_params<<<(L + 255) / 256, 256, 0, s>>>(d, len, u, kappa, beta, cost, phi, psi, w, head, opt->dn, opt->eps_tag);
    const int ne = std::max(n_lo, L);
    k_choice_info<<<(ne + 255) / 256, 256, 0, s>>>(d, lo_idx, n_lo, no_idx, L);
    const int nmax = std::max(std::max(L, V), std::max(N, 4));
    k_reset<<<(nmax + 255) / 256, 256, 0, s>>>(d, fifo_beg);
    const size_t smem = (size_t)smax * sizeof(float);
    if (raise_smem_attr(k_step_a, g_attr_a, opt->device, smem) != cudaSuccess) return SIM_ECUDA;
    for (int t = 0; t < T; ++t) {
        k_step_a<<<nblk, kBlockA, smem, s>>>(d, t, 0);
        k_step_b<<<(L + V + 255) / 256, 256, 0, s>>>(d, t);
    }
    k_step_a<<<nblk, kBlockA, smem, s>>>(d, T, 1);
    if (cudaGetLastError() != cudaSuccess) return SIM_ECUDA;
    // ---- outputs ----
    const cudaMemcpyKind k = out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t nbl = (size_t)nb * L;
    if (out->counts && cudaMemcpyAsync(out->counts, d.out_counts, nbl * sizeof(int), k, s) != cudaSuccess) return SIM_ECUDA;
    if (out->speed && cudaMemcpyAsync(out->speed, d.out_speed, nbl * sizeof(float), k, s) != cudaSuccess) return SIM_ECUDA;
    if (out->travel_time && cudaMemcpyAsync(out->travel_time, d.out_tt, nbl * sizeof(float), k, s) != cudaSuccess) return SIM_ECUDA;
    int err[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(err, d.err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SIM_ECUDA;
    if (out->n_waiting || out->n_on || out->n_arrived) {
        if (cudaMemcpyAsync(hs_counters, d.step_delta, (size_t)4 * T * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SIM_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return SIM_ECUDA;
    if (out->n_waiting || out->n_on || out->n_arrived) {
        int64_t nw = N, na = 0;
        for (int t = 0; t <= T; ++t) {
            if (t > 0) { nw -= hs_counters[4 * (t - 1)]; na += hs_counters[4 * (t - 1) + 1]; }
            if (out->n_waiting) out->n_waiting[t] = nw;
            if (out->n_arrived) out->n_arrived[t] = na;
            if (out->n_on) out->n_on[t] = N - nw - na;
        }
    }
    return err[0] ? err[0] : SIM_OK;
}
