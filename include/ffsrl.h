/*
 * ffsrl.h - C ABI of the GB300-native batched XPBD tissue simulator.
 *
 * The simulator advances many independent surgical-tissue environments at
 * once with the method of FF-SRL (Dall'Alba et al., arXiv 2503.18616):
 * extended position-based dynamics with substepping (Sec. III-A, Algorithm 1),
 * edge-distance constraints (Eq. 1) and tet-volume constraints (Eqs. 2-3) in
 * their compliance (XPBD) form, a kinematic tool that pushes tissue out of its
 * signed-distance volume (Sec. III-A "Collisions"), and the reinforcement-
 * learning interface of Sec. III-B: actions applied once per step, then
 * observations, reward (Sec. IV) and termination flags. Every variable of every
 * environment lives in one device array (Sec. III-B, last paragraph).
 *
 * Conventions for every entry point:
 *   - Return value: FFSRL_OK (0) on success, a negative FFSRL_E_* code
 *     otherwise; ffsrl_last_error() then gives a message (thread-local).
 *   - Pointers named *_dev are device pointers (for example the data of a
 *     torch CUDA tensor); they are read and written in stream order on the
 *     stream given to ffsrl_create, and the library never frees them. Pointers
 *     named *_host are ordinary host memory; calls taking them synchronise.
 *   - ffsrl_create deep-copies every host input. The library owns all of its
 *     device memory and frees it in ffsrl_destroy.
 *   - Kernels run asynchronously: a device-side error (non-finite positions)
 *     is reported by the next ffsrl_sync (FFSRL_E_NAN).
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns FFSRL_E_CUDA.
 *   - Layouts: "packed" vertex arrays hold env 0's vertices, then env 1's, and
 *     so on ([total_verts][3], float32, metres); per-env arrays are
 *     [n_env][...] in env order.
 */
#ifndef FFSRL_H
#define FFSRL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFSRL_OK 0
#define FFSRL_E_INVAL (-1)      /* bad argument or mesh */
#define FFSRL_E_CUDA (-2)       /* CUDA runtime error or no device */
#define FFSRL_E_OOM (-3)        /* device or host allocation failed */
#define FFSRL_E_DEGENERATE (-4) /* zero-volume tet or zero-length edge */
#define FFSRL_E_NAN (-5)        /* non-finite state detected on the device */
#define FFSRL_E_TIMEOUT (-6)    /* a bounded device wait gave up */

typedef struct ffsrl_sim ffsrl_sim; /* opaque */

/* One tet mesh in its rest state (Sec. III-A: V vertices with masses, tets).
 * Edges (distance constraints) are every tet edge; rest lengths and rest
 * volumes are computed from rest_pos before the loop (Eq. 1, Eq. 2). */
typedef struct {
    int32_t n_verts;         /* V, 1 .. 65535 */
    int32_t n_tets;          /* T, >= 1 */
    const double* rest_pos;  /* host [V][3], metres (rounded to float32 inside) */
    const double* inv_mass;  /* host [V], 1/m; 0 pins the vertex */
    const int32_t* tets;     /* host [T][4] vertex ids; a tet with negative
                                rest volume gets its last two ids swapped */
} ffsrl_mesh;

/* Method and task parameters. Lengths in metres, times in seconds. */
typedef struct {
    double dt;                /* simulation step Delta t (Algorithm 1) */
    int32_t substeps;         /* n substeps per step, h = dt / substeps (Sec. III-A) */
    int32_t iterations;       /* constraint iterations per substep (>= 0) */
    double gravity[3];        /* g of Algorithm 1 */
    double compliance_dist;   /* XPBD compliance alpha of edge constraints */
    double compliance_vol;    /* XPBD compliance alpha of volume constraints */
    double tool_radius;       /* radius of the sphere tool proxy */
    double action_scale;      /* tool displacement per step for a unit action */
    double tool_margin_xy;    /* tool box: rest bbox grown by this in x and y, */
    double tool_margin_below; /*   z from (top - below) ...                   */
    double tool_margin_above; /*   ... to (top + above)                       */
    double w_l, w_d, w_s;     /* reward weights of R = w_l l + w_d d + w_s s (Sec. IV) */
    double success_dist;      /* s = 1 when l < success_dist (3 mm in Sec. IV) */
    int32_t n_obs_verts;      /* sampled top-surface vertices in the observation */
    int32_t max_steps;        /* done when the step count reaches this (0 = never) */
    int32_t block_threads;    /* CUDA threads per environment (128, 256, 384, 512
                                 or 1024); 0 = autotuned (256 when forced) */
    int32_t schedule_flags;   /* 0 = autotuned; else FFSRL_SCHED_* bits forcing a schedule */
    int32_t solver;           /* FFSRL_SOLVER_*: colour Gauss-Seidel (0, the default) or the
                                 paper's Jacobi iterations with averaging (1, Sec. III-A) */
    int32_t auto_reset;       /* 1: an env whose step reported done starts its next episode at
                                 its next step (rest state, draws of the episode's seed
                                 splitmix64_nth(seed, 2^40 + k) for episode k >= 1) */
    int32_t tool_model;       /* FFSRL_TOOL_*: a sphere proxy (0, the default) or the paper's
                                 grasper (1, Sec. III-A): a shaft capsule from the remote centre
                                 of motion (rcm_height above the centre of the top face) to the
                                 tool point and two clamp capsules leaving the tool point at
                                 +-clamp_angle from the shaft axis, against the surface faces */
    int32_t reserved;         /* must be zero */
    double rcm_height;        /* grasper: remote centre of motion above the top face */
    double shaft_radius;      /* grasper: shaft capsule radius */
    double clamp_length;      /* grasper: clamp capsule length */
    double clamp_radius;      /* grasper: clamp capsule radius */
    double clamp_angle;       /* grasper: clamp opening angle from the shaft axis at reset, radians */
    double grasp_radius;      /* grasper: clamps closed below 3 degrees grasp the nearest free
                                 vertex within this distance of the dragging point (the clamp end,
                                 clamp_length beyond the tool point along the shaft) and keep it at
                                 its grasp-time distance (Sec. III-A dragging); opening releases */
    double conn_radius;       /* > 0: tissue connections (Sec. III-A) between the objects of a mesh
                                 (connected components of its tets, numbered by lowest vertex):
                                 every vertex of a surface face connects to the surface face of a
                                 lower object whose centroid is nearest at rest, if within this
                                 distance; a distance constraint keeps the vertex at its rest
                                 distance from the centroid, compliance compliance_dist, projected
                                 after the volume colours of each iteration. Gauss-Seidel only; no
                                 warm-start or recording step with connections */
} ffsrl_params;

#define FFSRL_TOOL_SPHERE 0
#define FFSRL_TOOL_GRASPER 1

#define FFSRL_SOLVER_GAUSS_SEIDEL 0
#define FFSRL_SOLVER_JACOBI 1

/* schedule_flags bits (execution choices only: results do not depend on them
 * beyond float32 rounding order, and not at all for the first three). */
#define FFSRL_SCHED_FORCE 1       /* use the bits below instead of autotuning them */
#define FFSRL_SCHED_NO_PERMUTE 2  /* keep vertex order in shared memory, colour order of records */
#define FFSRL_SCHED_NO_RING 4     /* read constraint records from L2 instead of the TMA ring */
#define FFSRL_SCHED_ENVS2 8       /* two envs per CTA sharing one ring (else one) */
#define FFSRL_SCHED_ENVS4 16      /* four envs per CTA sharing one ring */
#define FFSRL_SCHED_SURROGATE_PIPELINE 32  /* warm-start step as per-substep launches (features,
                                              network, substep) instead of one fused kernel */
#define FFSRL_SCHED_NO_CLUSTER 64  /* meshes above one CTA's shared memory use the global-memory
                                      working copy instead of a thread-block cluster */
#define FFSRL_SCHED_FOUR_CTAS 128  /* with FFSRL_SCHED_FORCE: the 256-thread, one-env, resident, ring
                                      kernel with registers budgeted for four CTAs per SM (64 per
                                      thread); FFSRL_E_INVAL where four CTAs do not fit an SM */
#define FFSRL_SCHED_WARM_STAGED 256  /* fused warm-start step: the kernel that stages the network's
                                        input tiles and corrections in global memory, instead of the
                                        one that builds each tile's input just in time (the default
                                        where a mesh's 1-ring spans at most four 128-row tiles) */
#define FFSRL_SCHED_GLOBAL_MEMORY 512  /* every env of the plain step on the global-memory working copy
                                          (the variant of meshes above the shared memory), even where
                                          its positions fit on chip: the streaming design point */

/* Sizes of a created simulator. */
typedef struct {
    int32_t n_env;
    int32_t n_meshes;
    int32_t obs_dim;          /* 3 + 3 * n_obs_verts */
    int32_t max_verts;        /* largest V over the meshes */
    int64_t total_verts;      /* sum over envs of their mesh's V (packed rows) */
    int32_t block_threads;    /* CUDA threads per env in use (largest group) */
    int32_t resident_envs;    /* envs whose state stays in shared memory */
    int32_t n_groups;         /* step-kernel launches per step */
    int32_t ring_envs;        /* envs whose constraint records stream through the TMA ring */
    int32_t envs_per_cta;     /* envs sharing one CTA (largest group) */
    int32_t ctas_per_sm;      /* CTAs per SM the step kernel's registers are budgeted for (largest group) */
} ffsrl_info;

/* Creates n_env environments; env e uses meshes[env_mesh[e]] (env_mesh NULL:
 * all use mesh 0) and the edge compliance env_compliance_dist[e] (NULL: the
 * params value). Builds every mesh's constraint tables (edges, rest values,
 * greedy first-fit colouring, colour-major order), allocates the device state
 * on cuda_stream (a cudaStream_t; NULL = the legacy default stream) and resets
 * every env with seed 0. On failure *out is NULL. */
int ffsrl_create(const ffsrl_mesh* meshes, int32_t n_meshes, const int32_t* env_mesh,
                 const double* env_compliance_dist, int32_t n_env, const ffsrl_params* params,
                 void* cuda_stream, ffsrl_sim** out);

/* Episode reset (Sec. III-B): for every env whose env_mask_dev[e] is nonzero
 * (env_mask_dev NULL: all envs) the positions return to rest, velocities to
 * zero, the tool to its start above the top face, the step count to zero, and
 * the observed vertices and target vertex are drawn from (seed, env). */
int ffsrl_reset(ffsrl_sim* sim, const uint8_t* env_mask_dev, uint64_t seed);

/* One simulation step of every env (Algorithm 1 with the substep loop):
 * tool update from actions_dev [n_env][3] in [-1, 1] (NULL: counter-based
 * device draws from each env's reset seed), then `substeps` substeps of
 * predict, coloured constraint projection, tool collision and velocity
 * update, then obs_dev [n_env][obs_dim], reward_dev [n_env] and done_dev
 * [n_env] (any of the three may be NULL). Asynchronous. */
int ffsrl_step(ffsrl_sim* sim, const float* actions_dev, float* obs_dev, float* reward_dev,
               uint8_t* done_dev);

/* ffsrl_step with host buffers: copies actions_host in, runs the step, copies
 * the outputs back and waits for them. Page-locked caller buffers
 * (cudaHostAlloc or registered) are copied directly; others go through
 * page-locked staging buffers owned by sim. */
int ffsrl_step_host(ffsrl_sim* sim, const float* actions_host, float* obs_host,
                    float* reward_host, uint8_t* done_host);

/* Waits for the sim's stream; returns FFSRL_E_NAN if any env produced a
 * non-finite position since the last call (and clears the flag). */
int ffsrl_sync(ffsrl_sim* sim);

int ffsrl_destroy(ffsrl_sim* sim);

int ffsrl_get_info(const ffsrl_sim* sim, ffsrl_info* out);

/* Thread-local message of the last failed call on this thread. */
const char* ffsrl_last_error(void);

/* Global env ids of the counter-based draws (Sec. III-B: envs are independent
 * slices of one batch, so a batch split across processes or GPUs is the same
 * set of envs): every draw of env e (actions when the step is given none,
 * observed vertices, target vertex, auto-reset episodes) is made for id
 * ids_host[e] instead of e. ids_host [n_env] int64 host array, each in
 * [0, 2^40) (NULL restores the default ids 0 .. n_env-1); ids need not be
 * distinct or sorted. A shard that holds envs 10..19 of a 1-process run with
 * ids 10..19 then draws exactly what that run draws for them. Takes effect for
 * draws made after the call: call it before ffsrl_reset. Synchronises. */
int ffsrl_set_env_ids(ffsrl_sim* sim, const int64_t* ids_host);

/* --- state access (checkpoint / resume, tests) ----------------------------- */

/* Packed state: x_dev, v_dev [total_verts][3]; tool_dev [n_env][3] float64.
 * Any pointer may be NULL. get writes them, set reads them. */
int ffsrl_get_state(ffsrl_sim* sim, float* x_dev, float* v_dev, double* tool_dev);
int ffsrl_set_state(ffsrl_sim* sim, const float* x_dev, const float* v_dev, const double* tool_dev);

/* Constraint tables of mesh `mesh` as built by ffsrl_create, copied to host.
 * which: 0 oriented tets [T][4], 1 flipped [T], 2 edges [E][2] (min,max),
 * 3 edge colour [E], 4 tet colour [T], 5 edge colour-major order [E],
 * 6 tet colour-major order [T], 7 edge colour offsets [n_ecol+1],
 * 8 tet colour offsets [n_tcol+1], 9 top-face vertices [n_top],
 * 10 surface faces [F][3] (ascending triples with a free vertex),
 * 11 their opposite tet vertices [F], 12 face colour-major order [F],
 * 13 face colour offsets [n_fcol+1], 14 tissue connections [C][4] (vertex,
 * then the face's ascending triple), 15 connection colour-major order [C],
 * 16 connection colour offsets [n_ccol+1], 17 object of each vertex [V].
 * With out_host NULL only *count is written (number of int32 values). */
int ffsrl_get_mesh_table(const ffsrl_sim* sim, int32_t mesh, int32_t which, int32_t* out_host,
                         int64_t* count);

/* Per-env integers copied to host (waits for the stream): step count,
 * target vertex, observed vertex ids [n_obs_verts], number of tool contacts
 * in the last substep and their vertex ids in ascending order.
 * contacts_host has room for the env's V entries; any pointer may be NULL. */
int ffsrl_get_env_ints(ffsrl_sim* sim, int32_t env, int32_t* step_count, int32_t* target,
                       int32_t* obs_ids_host, int32_t* n_contacts, int32_t* contacts_host);

/* --- learned warm-start network (not in the paper; a per-vertex
 *     15-64-64-3 ReLU perceptron, BF16 weights and activations, FP32
 *     accumulation, run on the tensor cores) --------------------------------- */

#define FFSRL_NET_PARAMS 5379  /* W1[64][15], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] */
#define FFSRL_NET_NORM 36      /* in_mean[15], in_std[15], out_mean[3], out_std[3] */

/* Installs the network: params_host [FFSRL_NET_PARAMS] float32 master weights
 * (rounded to BF16 inside), norm_host [FFSRL_NET_NORM] the frozen feature and
 * output normalisation (std > 0). Host buffers; the call copies them. */
int ffsrl_set_network(ffsrl_sim* sim, const float* params_host, const float* norm_host);

/* Copies the float32 master parameters (as ffsrl_set_network takes them) to params_host. */
int ffsrl_get_network(const ffsrl_sim* sim, float* params_host);

/* Gradient of the weighted mean squared error of the network on a batch,
 * L = sum_r w_r |y_r - t_r|^2 / (3 weight_sum) in normalised output units
 * (t_r = (target_r - out_mean) / out_std), computed on the tensor cores with
 * BF16 operands: features_dev [rows][16] raw features, targets_dev [rows][4]
 * raw targets (x, y, z, ignored), row_weight_dev [rows] float32 weights,
 * weight_sum their sum. grad_dev [FFSRL_NET_PARAMS] (may be NULL) receives the
 * gradient in the layout of the parameters, loss_dev [1] (may be NULL) the
 * weighted sum of squared errors. Asynchronous. */
int ffsrl_network_gradient(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                           const float* row_weight_dev, int64_t rows, float weight_sum, float* grad_dev,
                           float* loss_dev);

/* One Adam step (Kingma & Ba 2015; beta 0.9, 0.999, eps 1e-8) of the float32
 * master parameters on the gradient of that loss, then re-rounds the BF16
 * copies the network runs with. loss_dev as above. Asynchronous. */
int ffsrl_train_network(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                        const float* row_weight_dev, int64_t rows, float weight_sum, float lr, float* loss_dev);

/* One Adam step (as in ffsrl_train_network) on a caller-given gradient:
 * grad_dev [FFSRL_NET_PARAMS] float32 device array in the layout of the
 * parameters (for example the sum over data-parallel ranks of their
 * ffsrl_network_gradient results, divided by the rank count), then re-rounds
 * the BF16 copies. The step count t of the bias correction is the number of
 * Adam steps since ffsrl_set_network. Asynchronous; grad_dev must stay valid
 * until the stream has passed the call. */
int ffsrl_network_adam_step(ffsrl_sim* sim, const float* grad_dev, float lr);

/* Frozen normalisation of a training batch, computed on the device in
 * double: over the rows r < rows with row_weight_dev[r] > 0, per feature
 * column (features_dev [rows][16], the 16th ignored) and per target column
 * (targets_dev [rows][4], the 4th ignored) the mean and the population
 * standard deviation (divisor = number of such rows; 1 where a column has no
 * spread). norm_host [FFSRL_NET_NORM] float32 receives in_mean[15],
 * in_std[15], out_mean[3], out_std[3], the layout ffsrl_set_network takes.
 * Synchronises. FFSRL_E_INVAL if no row has a positive weight, FFSRL_E_NAN
 * if a selected value is not finite. No network needs to be installed. */
int ffsrl_network_normalisation(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                                const float* row_weight_dev, int64_t rows, float* norm_host);

/* out_dev[r] = (network output of features_dev[r], 0) for r < rows:
 * features_dev [rows][16] float32 raw features (the 16th is ignored), output
 * [rows][4] float32 de-normalised (x, y, z, 0). Asynchronous on the sim's
 * stream; a tensor-core completion timeout is reported by ffsrl_sync
 * (FFSRL_E_TIMEOUT). */
int ffsrl_network_forward(ffsrl_sim* sim, const float* features_dev, float* out_dev, int64_t rows);

/* Surrogate-assisted step of every env (the warm-start; requires a network):
 * per substep, predict (Algorithm 1), add the network's correction to free
 * vertices, run one constraint iteration, and if the largest relative
 * constraint violation of the env (|C|/d for edges, |C|/|V0| for tets) exceeds
 * `threshold`, restore the prediction and run `n_full` iterations instead;
 * then collision and velocity update. Outputs as ffsrl_step; fallbacks_dev
 * [n_env] int32 (may be NULL) is incremented once per fallen-back substep;
 * residual_dev [n_env] float32 (may be NULL) is raised to the largest checked
 * residual (the caller initialises it, e.g. to zero). A threshold of +inf
 * never falls back (the residual is then evaluated only for residual_dev);
 * any other threshold falls back unless the residual is at most the
 * threshold, so a NaN residual falls back. Asynchronous. */
int ffsrl_step_surrogate(ffsrl_sim* sim, const float* actions_dev, float* obs_dev, float* reward_dev,
                         uint8_t* done_dev, double threshold, int32_t n_full, int32_t* fallbacks_dev,
                         float* residual_dev);
/* Implementation note: envs whose mesh fits one CTA's shared memory take the
 * whole step in one fused kernel (state resident on chip, the network on the
 * tensor cores of the same CTA); larger meshes, or every mesh when
 * FFSRL_SCHED_SURROGATE_PIPELINE is set, take three launches per substep
 * (features, network, substep). Both compute the same operations. */

/* Mixed rollout: from the next ffsrl_step (and ffsrl_step_host) on, the envs
 * whose byte in mask_host [n_env] is non-zero take the surrogate-assisted step
 * of ffsrl_step_surrogate (same threshold and n_full semantics), the others
 * the plain step, both within the one call and without a host round trip.
 * mask_host NULL switches back to plain stepping for every env. fallbacks_dev
 * (may be NULL) is caller-owned int32 [n_env], incremented per fallen-back
 * substep for as long as the setting lasts. Requires a network
 * (ffsrl_set_network) and meshes that fit the fused kernel (FFSRL_E_INVAL
 * otherwise). The mask is copied; ffsrl_step_noalloc rejects a sim in this
 * mode. */
int ffsrl_set_surrogate_envs(ffsrl_sim* sim, const uint8_t* mask_host, double threshold, int32_t n_full,
                             int32_t* fallbacks_dev);

/* Grasper clamp openings (radians) from the next step on: angles_dev [n_env]
 * float32 device array, read by a kernel on the sim's stream (asynchronous:
 * keep it valid until the stream has passed the call). Below 3
 * degrees the clamps count as closed and grasp (ffsrl_params.grasp_radius).
 * Reset restores ffsrl_params.clamp_angle. FFSRL_E_INVAL without the grasper. */
int ffsrl_set_clamp_angles(ffsrl_sim* sim, const float* angles_dev);

/* Grasped vertex of every env (-1: none) into grasp_host [n_env]; synchronises. */
int ffsrl_get_grasp(ffsrl_sim* sim, int32_t* grasp_host);

/* Plain step with `n_full` iterations per substep that records training data:
 * features_dev [substeps][rows][16] (features of every vertex row at each
 * substep's prediction) and targets_dev [substeps][rows][4] (positions after
 * the solve minus the prediction, before collision), either may be NULL.
 * residual_dev [n_env] (may be NULL) is raised to the largest residual the
 * solve leaves. Rows: ffsrl_get_rows. */
int ffsrl_record_step(ffsrl_sim* sim, const float* actions_dev, int32_t n_full, float* features_dev,
                      float* targets_dev, float* residual_dev);

/* Row layout of per-vertex buffers: *n_rows rows; env e's vertices occupy
 * rows row_off_host[e] .. row_off_host[e] + V_e - 1 (row_off_host [n_env] or NULL). */
int ffsrl_get_rows(const ffsrl_sim* sim, int64_t* n_rows, int32_t* row_off_host);

/* --- allocation-free step (no counterpart in the paper) ------------------- */

/* Size of the static device scratch array used by ffsrl_step_noalloc. */
#define FFSRL_NOALLOC_SCRATCH_BYTES (32u << 20)

/* One simulation step of caller-owned states that allocates no memory.
 *
 * Who needs it: callers that must not call cudaMalloc or cudaFree while they
 * step the simulation - for example a real-time control loop, where those
 * calls can synchronise the whole device and stall for milliseconds, a
 * process whose device memory is reserved up front by another allocator
 * (a deep-learning framework's caching allocator), so a further cudaMalloc
 * fails or fragments memory, or a plugin host that forbids allocation inside
 * its per-step callback. Such a caller creates the simulator once, where it
 * may allocate, and then steps states it owns itself with this call.
 *
 * What it does: advances every env of `sim` by one step exactly as ffsrl_step
 * does (same kernels, same schedule, same results), but on the state in the
 * caller's arrays instead of the sim's own state: x_dev and v_dev are packed
 * [total_verts][3] float32 positions and velocities, tool_dev is [n_env][3]
 * float64 tool centres; all three are read and overwritten in place.
 * actions_dev [n_env][3] is required (caller-owned state has no step counter
 * for device-drawn actions). No observation, reward or done flags are
 * produced. The sim's own state is neither read nor changed; only its
 * constraint tables, parameters and schedule are used. A device error of the
 * call (non-finite positions, a bounded wait that gave up) is recorded in the
 * sim's error flags, so the next ffsrl_sync reports it. Sims with the grasper
 * tool (whose grasp is per-sim state), auto-reset or a mixed rollout are
 * refused with FFSRL_E_INVAL. Asynchronous on the sim's stream.
 *
 * Scratch: the working copies of the state, the substep-start positions, the
 * per-env counters and done flags and (with iterations > 1) the Lagrange
 * multipliers live in
 * one file-scope static device array of FFSRL_NOALLOC_SCRATCH_BYTES (32 MiB),
 * which every GPU that loads the library holds until the process exits. A sim
 * whose scratch would exceed it (about 36 B per padded vertex row plus 13 B per
 * env, more with iterations > 1 or meshes too large for shared memory) is
 * rejected with FFSRL_E_INVAL and a message giving both sizes; for the
 * 2601-vertex block that is about 340 envs. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. Every call shares the one
 * array and it keeps the last call's contents: the call clears what must start
 * at zero, and calls that overlap on the GPU (two streams, two sims, two
 * threads) race on it and must be ordered by the caller. The call never
 * allocates or frees device or pinned host memory. */
int ffsrl_step_noalloc(ffsrl_sim* sim, const float* actions_dev, float* x_dev, float* v_dev,
                       double* tool_dev);

#ifdef __cplusplus
}
#endif

#endif /* FFSRL_H */
