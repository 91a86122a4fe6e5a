/*
 * trafficsim.h -- C ABI of the B300 (sm_103a) differentiable agent-based traffic
 * simulator (Makinoshima et al., "Ultra-fast Traffic Nowcasting and Control via
 * Differentiable Agent-based Simulation").
 *
 * One simulator step is phi = g o f (Results, "Differentiable agent-based traffic
 * simulation"): f is Newell's car-following update applied to every vehicle of
 * every link (Methods Eq. newell_model; SI-A), g is the node model that lets the
 * leading vehicle of a link choose its next link with a Gumbel-softmax /
 * straight-through sample (SI-B "Link choice", Eqs. softmax, gumbel,
 * straigththrough), resolves competing entrants by a second Gumbel sample over
 * merge priorities (SI-B "Merge choice") and transfers the winners with
 * trajectory grafting (SI-B Eq. transfer; SI-C).  Link counts at the midpoint
 * follow SI-D.  The reverse-mode adjoint is that of the straight-through /
 * trajectory-grafting surrogate the paper differentiates with jax.grad (Methods,
 * "Optimization").
 *
 * Conventions
 *  - All sizes are int32 unless noted; all real data is float32.
 *  - Arrays passed to sim_create / sim_set_params are HOST pointers owned by the
 *    caller; the library copies them and keeps no reference.
 *  - The handle owns every device buffer it allocates (cudaMalloc) and frees
 *    them in sim_destroy.
 *  - Output buffers belong to the caller; `on_device` says whether they are
 *    device pointers (written asynchronously on the handle's stream) or host
 *    pointers (the call returns after the copy).
 *  - All device work is enqueued on the handle's stream: the caller's
 *    `sim_options.stream` if non-NULL, else a stream the handle creates.
 *  - Every call returns SIM_OK (0) or a SIM_E* code; sim_last_error() gives the
 *    text.  No call aborts the process; device-side failures (queue overflow,
 *    route-log overflow, bounded waits) are reported through an error word,
 *    never by trapping the GPU.
 *  - A handle is not thread safe; distinct handles are independent.
 */
#ifndef TRAFFICSIM_H
#define TRAFFICSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SIM_API __attribute__((visibility("default")))
#else
#define SIM_API
#endif

#define SIM_OK        0
#define SIM_EINVAL    1   /* bad argument, shape, index or network          */
#define SIM_ENOMEM    2   /* device allocation failed                        */
#define SIM_ECUDA     3   /* CUDA runtime error                              */
#define SIM_ETIMEOUT  4   /* a bounded device wait expired                   */
#define SIM_ESTATE    5   /* call not valid in the handle's current state    */
#define SIM_EOVERFLOW 6   /* a fixed-capacity device buffer would overflow   */

/* Fixed point of the outflow credit: one vehicle = 65536 units. */
#define SIM_FX_ONE 65536

typedef struct sim_ctx *sim_handle;

/* Road network (SI-A, SI-B).  Links are directed tail -> head.
 * q_fx: outflow credit added per step, in 1/65536 vehicle (capacity q * dt).
 * phi, psi: [L * F] row-major link features; the utility of turning into link m
 *   for a vehicle bound for zone z is  beta_m / cost_m + sum_f w_f phi[m,f]
 *   + (sum_f w_f psi[m,f]) * dest_feat[z, head_m]   (SI-B Eq. for V, with the
 *   origin/destination factors the text allows).
 * node_zone: [V] destination zone of each node; dest_feat: [Z * V]. */
typedef struct {
    int32_t V, L;
    const int32_t *tail, *head;
    const float *length;
    const int32_t *q_fx;
    int32_t F;
    const float *phi, *psi;
    int32_t Z;
    const int32_t *node_zone;
    const float *dest_feat;
} sim_network;

/* Travel demand: vehicle i joins the queue of its origin node at step
 * dep_step[i] and leaves the network on reaching any node of dest_zone[i].
 * od[i] in [0, n_od) groups vehicles by OD demand parameter od_lambda. */
typedef struct {
    int32_t N;
    const int32_t *origin, *dest_zone, *dep_step, *od;
    int32_t n_od;
    const float *od_lambda;
} sim_demand;

/* Differentiable parameters (Methods "Experimental setting"): per link free
 * speed u (m/s), jam density kappa (veh/m), merge priority alpha, cost
 * sensitivity beta and cost c; route-choice coefficients w [F]; merge priority
 * of the origin queues. */
typedef struct {
    const float *u, *kappa, *alpha, *beta, *cost;
    const float *w;
    float alpha_origin;
} sim_params;

/* Run options.  dt = tau * dn with tau = 1 (Methods, Eq. newell_model); M is the
 * sentinel of SI-A (99999); eps_arr the arrival tolerance of Alg. S2 (1e-2 m);
 * eps_tag the relative dead band that tags ties of the car-following min/max for
 * the adjoint; tau_gumbel the Gumbel-softmax temperature (Eq. gumbel).
 * Random numbers: Philox4x32-10 keyed by (seed, scenario_id), counter
 * (vehicle, step, stream, block).  obs_every: steps per observation bin.
 * ckpt_every: steps between checkpoints kept for sim_backward (0 = forward only).
 * route_cap: entries of the per-vehicle route log (needed by sim_backward). */
typedef struct {
    float dt, dn, tau_gumbel, M, eps_arr, eps_tag;
    uint64_t seed;
    uint32_t scenario_id;
    int32_t obs_every;
    int32_t ckpt_every;
    int32_t route_cap;
    int32_t device;
    void *stream;          /* cudaStream_t or NULL */
} sim_options;

/* Rollout outputs, n_bins = ceil(T / obs_every) bins of obs_every steps:
 * counts[b*L + j]      vehicles passing the midpoint of link j in bin b (SI-D);
 * speed[b*L + j]       mean speed on link j in bin b (distance / vehicle-time);
 * travel_time[b*L + j] mean link time of the vehicles leaving j in bin b;
 * n_waiting/n_on/n_arrived[t], t = 0..T: vehicles not yet on the network, on a
 * link, and arrived.  Any pointer may be NULL. */
typedef struct {
    int32_t *counts;
    float *speed, *travel_time;
    int64_t *n_waiting, *n_on, *n_arrived;
    int32_t on_device;
} sim_outputs;

/* Gradients of a scalar loss (sim_backward).  Any pointer may be NULL. */
typedef struct {
    float *d_u, *d_kappa, *d_alpha, *d_beta, *d_cost;   /* [L] */
    float *d_w;                                         /* [F] */
    float *d_alpha_origin;                              /* [1] */
    float *d_od_lambda;                                 /* [n_od] */
    int32_t on_device;
} sim_grads;

/* Exported state (host buffers, any may be NULL): per vehicle its link (-1 not
 * yet on the network, -2 arrived), position, rank in its link queue (0 = the
 * leader; -1 off-network) and entry step (-1 off-network); per link the outflow credit and
 * cumulative exits; per node the number of vehicles its origin queue released. */
typedef struct {
    int32_t *veh_link;
    double *veh_pos;
    int32_t *veh_rank, *veh_entry;
    int64_t *link_credit, *link_exits;
    int32_t *fifo_off;
} sim_state_view;

/* Decisions of the last step (host buffers, any may be NULL): candidate vehicle
 * and target per link / origin node (-1 none, -2 leaves to its destination,
 * -3 chosen link not vacant), and the vehicle that entered each link (-1 none). */
typedef struct {
    int32_t *link_cand, *link_target, *node_cand, *node_target, *link_in;
} sim_records;

/* Number of observation bins of a T-step rollout. */
SIM_API int32_t sim_n_bins(int32_t T, int32_t obs_every);

/* Create a simulator on options->device.  Validates the network (indices,
 * choice sets of at most 32 links, positive lengths / capacities / costs),
 * copies every input to the device and leaves the handle at t = 0.
 * Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA.  *out is NULL on failure. */
SIM_API int sim_create(const sim_network *net, const sim_demand *dem, const sim_params *par,
               const sim_options *opt, sim_handle *out);

/* Replace the differentiable parameters (host arrays, same sizes as at create).
 * Takes effect at the next reset / rollout. */
SIM_API int sim_set_params(sim_handle h, const sim_params *par);

/* As sim_set_params, with the arrays (u, kappa, alpha, beta, cost [L], w [F])
 * and the origin queues' merge priority (*alpha_origin, one float; the struct's
 * alpha_origin field is not read) in memory of the handle's device, e.g.
 * tensors of a training loop.  The copies and the derivation of the per-link
 * quantities are enqueued on the handle's stream without a host
 * synchronisation: the arrays must hold their values until the stream reaches
 * the call (order the producer's stream before it with an event) and may
 * change after.  Validation (the rules of sim_set_params) runs on the device;
 * an invalid parameter is reported as SIM_EINVAL by the next call that reads
 * the handle's device errors (a rollout into host outputs, sim_step,
 * sim_backward), until parameters are set again.  The paper has no
 * counterpart.  Errors: SIM_EINVAL (NULL arrays), SIM_ECUDA. */
SIM_API int sim_set_params_device(sim_handle h, const sim_params *par, const float *alpha_origin);

/* Reset to t = 0 for a rollout of horizon T (every vehicle waiting, links empty,
 * full outflow credit).  Errors: SIM_EINVAL (T < 1). */
SIM_API int sim_reset(sim_handle h, int32_t T);

/* Advance n_steps steps of phi = g o f from the current time; the last step may
 * not pass the horizon given to sim_reset.  Observation bins close as they
 * complete.  Errors: SIM_ESTATE (beyond horizon / no reset), SIM_EOVERFLOW. */
SIM_API int sim_step(sim_handle h, int32_t n_steps);

/* Reset, run T steps, close the last observation bin and write the outputs.
 * With options.ckpt_every > 0 it also keeps the checkpoints and route log that
 * sim_backward needs.  The persistent executor runs the steps in one
 * cooperative launch (one per checkpoint segment with ckpt_every > 0); the
 * two-kernel executor replays them from a CUDA graph captured on the first
 * rollout of each horizon.  Errors: as sim_reset / sim_step, SIM_ECUDA. */
SIM_API int sim_rollout(sim_handle h, int32_t T, sim_outputs *out);

/* Copy the outputs of the current run (bins closed so far; counters up to the
 * current step) -- the rollout outputs when the run was driven by sim_step. */
SIM_API int sim_get_outputs(sim_handle h, sim_outputs *out);

/* Per-step counters of the current run: counters[4*t + k] for step t, k = 0
 * vehicles released by origin queues, 1 arrivals, 2 node-model candidates,
 * 3 link entries.  `counters` is a host array of 4 * (steps so far) int32. */
SIM_API int sim_step_counters(sim_handle h, int32_t *counters);

/* Instrumented rollout for measurement: the same kernels as sim_rollout,
 * launched one by one with a CUDA event recorded on the handle's stream before
 * and after every launch.  kernel_ms[k] receives the summed device time of
 * kernel class k (0 = node-model/car-following kernel, 1 = transfer kernel,
 * 2 = final observation) and launches[k] the launch counts.  Outputs as
 * sim_rollout. */
SIM_API int sim_profile_rollout(sim_handle h, int32_t T, sim_outputs *out, double *kernel_ms,
                                int64_t *launches);

/* Reverse-mode gradient of L = sum_{b,j} dL_dcounts[b,j] * counts[b,j] (+ the
 * optional terms below) through the straight-through / trajectory-grafting
 * surrogate of the last sim_rollout (SI-B, SI-C, SI-D), recomputing each
 * checkpoint segment.  dL_dcounts: [n_bins * L]; dL_dxT: optional [N] adjoint
 * of the final vehicle positions.  Inputs are host or device per on_device.
 * Errors: SIM_ESTATE (no rollout with ckpt_every > 0 since the last reset). */
SIM_API int sim_backward(sim_handle h, const float *dL_dcounts, const float *dL_dxT,
                 int32_t inputs_on_device, sim_grads *out);

/* Copy the current state / last-step decisions to host buffers. */
SIM_API int sim_get_state(sim_handle h, sim_state_view *out);

/* Replace the dynamic state by a given one at step t of the current horizon
 * (0 <= t <= T of the last sim_reset / sim_rollout), e.g. the oracle's state
 * after a flagged near-tie, so that a lockstep comparison can continue from
 * it.  *in holds host arrays in the layout of sim_state_view (every field
 * required): vehicle link (-1 waiting / not yet departed, -2 arrived),
 * position, rank in its queue (0 = leader), entry step; per link outflow
 * credit (2^-16 veh) and exits; per origin node the number of vehicles
 * released.  The next sim_step continues with step t.  The vacancy / arrival
 * flags of step t are derived from the queues as the step would derive them.
 * The observation bin containing t restarts at t (its counts, speeds and
 * travel times cover [t, bin end)); the step counters of earlier steps are
 * kept.  The paper has no counterpart (its state is a dense tensor one can
 * assign).  Errors: SIM_ESTATE (no sim_reset yet, t out of range), SIM_EINVAL
 * (a field out of range, ranks not 0..n-1 per link, a queue over capacity, a
 * position outside its link, waiting vehicles that do not match the origin
 * queues). */
SIM_API int sim_set_state(sim_handle h, const sim_state_view *in, int32_t t);
SIM_API int sim_get_records(sim_handle h, sim_records *out);

/* Launch shape of the node-model kernel: queue slots staged in shared memory
 * per link block (256..8192, default 2048; links are packed into blocks up to
 * this many slots).  Results do not depend on it.  Errors: SIM_EINVAL. */
SIM_API int sim_set_stage(sim_handle h, int32_t slots);

/* Forward executor of sim_rollout / sim_step (results are bit-identical):
 *   SIM_EXEC_STEP        two kernels per step (link blocks, then transfers),
 *                        captured into a CUDA graph per horizon;
 *   SIM_EXEC_PERSISTENT  the whole run in one cooperative launch, one CTA per
 *                        SM, every link queue resident in shared memory and one
 *                        grid-wide barrier per step (the paper has no
 *                        counterpart: its step is a sequence of XLA ops);
 *   SIM_EXEC_AUTO        (default) persistent when available, else step.
 * The persistent executor is available when every queue of the network fits in
 * the shared memory of the GPU's SMs.  For a handle that records the reverse-pass
 * tape (ckpt_every > 0) it runs sim_rollout as one launch per checkpoint segment
 * and the segment recomputation of sim_backward as one recording launch per
 * segment; sim_step of such a handle uses the two-kernel path.  Errors:
 * SIM_EINVAL (unknown value, or persistent requested where it is unavailable;
 * the text says why). */
#define SIM_EXEC_AUTO       0
#define SIM_EXEC_STEP       1
#define SIM_EXEC_PERSISTENT 2
SIM_API int sim_set_executor(sim_handle h, int32_t executor);
/* Executor the next forward run will use (SIM_EXEC_STEP or SIM_EXEC_PERSISTENT),
 * -1 for a NULL handle. */
SIM_API int32_t sim_get_executor(sim_handle h);

/* Work partition of the persistent executor.  Each CTA owns a run of
 * consecutive links; the runs are chosen so that the largest sum of link
 * weights over a run is as small as the shared-memory limits allow.  By
 * default a link weighs its queue capacity + 16 slots.  w (host, [L],
 * finite, >= 0, not all 0) replaces that by a relative weight per link, e.g.
 * the mean number of vehicles on the link measured in an earlier rollout plus
 * a per-link constant, so that CTAs get equal work rather than equal capacity.
 * NULL restores the default.  Results do not depend on the partition (they
 * are bit-identical).  Call between runs, not while another call on h is in
 * progress.  The paper has no counterpart (its step is not partitioned).
 * Errors: SIM_EINVAL (invalid weights; a weighting under which the queues no
 * longer fit leaves the previous partition in place). */
SIM_API int sim_set_partition_weights(sim_handle h, const float *w);
/* Number of CTAs of the persistent executor (0 if it is unavailable, -1 on
 * error); first_link (host, may be NULL) receives the G + 1 group bounds. */
SIM_API int32_t sim_persist_groups(sim_handle h, int32_t *first_link);

/* Test hook for the bounded waits of the persistent executor: the next
 * persistent launch of h waits at its grid barriers for `missing` arrivals
 * that never come, so every CTA gives up after its bounded wait (about 2 s),
 * the call reports SIM_ETIMEOUT and the device context stays usable; the
 * handle needs sim_reset (or sim_rollout) before it is used again.  No GPU
 * fault is involved: the wait simply runs out.  The paper has no counterpart.
 * Errors: SIM_EINVAL (missing < 0, or no persistent executor for h). */
SIM_API int sim_test_barrier_timeout(sim_handle h, int32_t missing);

/* The stream the handle's work is enqueued on (a cudaStream_t: the caller's
 * options.stream, or the one the handle created), NULL for a NULL handle.
 * Device outputs are complete once this stream has reached the point where
 * the call returned; callers on other streams order themselves after it with
 * an event.  The paper has no counterpart. */
SIM_API void *sim_get_stream(sim_handle h);

/* Move the handle's work to another stream of its device (the old stream is
 * drained first; a stream the handle created is destroyed).  NULL: only drain.
 * Not for a handle that is a member of a live batch. */
SIM_API int sim_set_stream(sim_handle h, void *stream);

/* Segment recomputation of the reverse pass (sim_backward):
 *   SIM_RECOMPUTE_SERIAL (default)  each segment is recomputed by one
 *       recording launch of the persistent executor just before its reverse
 *       kernels;
 *   SIM_RECOMPUTE_OVERLAP  segment s - 1 is recomputed by the two-kernel
 *       executor on a low-priority stream while the reverse kernels of
 *       segment s run on a high-priority one.
 * Both use two tape sets (by segment parity: the Jacobian kernel of a
 * segment reads its set while the next is recorded), about 2 x K x (1 byte per
 * queue slot + 68 bytes per link + 20 per origin queue), positions at bin ends
 * and the segment-start vehicle ids besides.  Both give the same tape, so the
 * same gradients (up to the order of the double-precision atomic additions).
 * SERIAL falls back to OVERLAP when the handle has no persistent executor.
 * Errors: SIM_EINVAL (unknown mode). */
#define SIM_RECOMPUTE_OVERLAP 0
#define SIM_RECOMPUTE_SERIAL  1
SIM_API int sim_set_recompute(sim_handle h, int32_t mode);

/* Device memory of simulators and batches comes from a stream-ordered memory
 * pool per device, which keeps freed blocks mapped for the next simulator (as
 * a caching allocator does); reverse-pass workspaces (one per sim_backward
 * running at the same time on the device) stay for reuse too.  This frees the
 * idle workspaces and returns the device's unused cached blocks to the
 * driver; memory of live simulators is unaffected.  It synchronises the
 * device.  Errors: SIM_EINVAL (device index), SIM_ECUDA. */
SIM_API int sim_release_cached_memory(int32_t device);

/* Current time step and device bytes held by the handle. */
SIM_API int32_t sim_time(sim_handle h);
SIM_API size_t sim_device_bytes(sim_handle h);

/* ---------------------------------------------------------------------------
 * Batches: many simulators advanced together, one launch per phase and step
 * for all of them.  Members keep their own network, demand, parameters, state,
 * step counter and horizon; results of a member are the same as when it runs
 * alone (its decisions depend on its own random key and state only).  While
 * batched, members use the batch's stream (that of the first member) and must
 * not be stepped, reset or reshaped through their own handles; their outputs,
 * state and sim_backward (after they finished) remain available.
 * ------------------------------------------------------------------------- */
typedef struct sim_batch_ctx *sim_batch;

/* Group n distinct handles of one device.  Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA. */
SIM_API int sim_batch_create(const sim_handle *members, int32_t n, sim_batch *out);

/* Reset member k for a rollout of horizon T; it joins at the next step boundary
 * of sim_batch_advance (continuous batching). */
SIM_API int sim_batch_start(sim_batch b, int32_t k, int32_t T);

/* Advance every running member by n_steps steps (a member reaching its horizon
 * closes its last bin in the following step and then stays idle).  finished:
 * optional [n] flags, 1 for members done with their horizon.  With the
 * persistent batch executor the n_steps steps are one cooperative launch;
 * with the step executor, runs of 8 or more steps are replayed from a CUDA
 * graph captured once per length.  Returns after the stream has drained.
 * Errors: a member's device error (its code), SIM_ETIMEOUT when a grid barrier
 * of the persistent launch gave up (the members' states are then undefined). */
SIM_API int sim_batch_advance(sim_batch b, int32_t n_steps, int32_t *finished);

/* Executor of the batch (SIM_EXEC_* above):
 *   SIM_EXEC_STEP        per step a checkpoint kernel, the link-block kernel, the
 *                        transfer kernel and a counter kernel over all members
 *                        (graph-captured);
 *   SIM_EXEC_PERSISTENT  one cooperative launch per advance, one CTA of 1,024
 *                        threads per SM; a warp takes 32 links (or 32 origin
 *                        nodes, or 32 transfer elements) of one member through
 *                        the node model, with a bounded grid barrier after the
 *                        node model and after the transfers of every step;
 *   SIM_EXEC_AUTO        (default) persistent when available, else step.
 * Both give every member bitwise the same outputs and state as its solo run.
 * Errors: SIM_EINVAL (unknown value; persistent requested but unavailable --
 * more than 1,024 members, or no cooperative launch on the device). */
SIM_API int sim_batch_set_executor(sim_batch b, int32_t executor);
SIM_API int32_t sim_batch_get_executor(sim_batch b);

/* Test hook of the persistent batch executor: every grid barrier of the next
 * sim_batch_advance waits for `missing` arrivals that never come, so its
 * bounded wait runs out (about 2 s); the advance reports SIM_ETIMEOUT.  The
 * running members' states are then undefined until sim_batch_start restarts
 * them.  No GPU fault is involved.  Errors: SIM_EINVAL (missing < 0, or no
 * persistent batch executor). */
SIM_API int sim_batch_test_barrier_timeout(sim_batch b, int32_t missing);

/* Start every member with horizon T and run all of them to the end. */
SIM_API int sim_batch_rollout(sim_batch b, int32_t T);

/* Release the batch (the member handles stay valid and get their streams back). */
SIM_API int sim_batch_destroy(sim_batch b);
SIM_API const char *sim_batch_last_error(sim_batch b);

/* Forward rollout that allocates nothing -- the same computation and outputs as
 * sim_create + sim_rollout + sim_destroy, for callers that may not allocate
 * device memory: plug-ins inside a host application whose memory manager owns
 * every device allocation (it may refuse, or fail to account for, a cudaMalloc
 * made behind its back), and real-time loops, where cudaMalloc / cudaFree can
 * block the host thread and synchronise the device.  The paper has no
 * counterpart of this entry point.
 *   Scratch: one file-scope device array of 16 MiB (every GPU that loads the
 *   library holds it until the process exits) plus fixed static host buffers.
 *   Limits: V <= 4096 nodes, L <= 8192 links, N <= 65536 vehicles, T <= 8192
 *   steps, all choice sets together <= 65536 entries, and every array of the
 *   run inside the 16 MiB; beyond them the call returns SIM_EOVERFLOW before
 *   any device work.
 *   Inputs: host arrays as for sim_create (phi, psi and w may be NULL only when
 *   F = 0; the demand arrays only when N = 0).  Outputs: as sim_rollout
 *   (device or host per out->on_device; the n_* counters only into host
 *   memory: with on_device set they must be NULL).
 *   Work runs on options->stream (NULL = the default stream) of
 *   options->device; the call returns after the stream has drained.
 *   The first call on a device looks up the device address of the scratch
 *   array (cudaGetSymbolAddress) before any work is enqueued.  Every call
 *   re-initialises the whole scratch (nothing of an earlier call is read).
 *   The static host buffers are guarded by one mutex, so calls from several
 *   host threads run one after another.  The device array is shared too: a
 *   call whose work still runs on the GPU when another call starts (on another
 *   stream, or issued by code that does not wait for it) races with it.
 *   Returns SIM_OK, SIM_EINVAL (bad or NULL argument), SIM_EOVERFLOW (a limit
 *   above, or a link queue overflowed on the device) or SIM_ECUDA; no error
 *   text is kept for this call. */
SIM_API int sim_rollout_static(const sim_network *net, const sim_demand *dem, const sim_params *par,
                               const sim_options *opt, int32_t T, sim_outputs *out);

/* Release every resource of the handle (NULL is accepted). */
SIM_API int sim_destroy(sim_handle h);

/* Text of the last error on this handle (or of the last failed sim_create when
 * h is NULL).  Valid until the next call on the handle. */
SIM_API const char *sim_last_error(sim_handle h);

#ifdef __cplusplus
}
#endif
#endif /* TRAFFICSIM_H */
