/*
 * mr_lbm.h -- C-ABI of the GB300 implementation of the fully adaptive
 * multiresolution lattice-Boltzmann time step of Bellotti, Gouarin, Graille
 * and Massot, "Multidimensional fully adaptive lattice Boltzmann methods with
 * error control based on multiresolution analysis" (arXiv 2103.02903).
 *
 * One call of mr_lbm_step() runs, entirely on the GPU, the loop body of
 * Algorithm 1 (Sec. 6.2): the multiresolution encode of the stored
 * post-collision field (projection, Def. Projection; prediction with s = 1,
 * Sec. 4.1; details, Def. Details; group norm, Sec. 4.4), the mesh adaptation
 * Lambda(t+dt) = G o H_eps o T_eps (Lambda(t)) (Eq. Thresholding,
 * Eq. AdditionNeigh, the refinement rule of Sec. 5.1, Def. Grading), the
 * data transfer to the new leaves (Sec. 5.1), the leaf-reconstruction
 * transport (Eq. AdaptiveAdvectionPhase evaluated with the flattened weights
 * of Eq. PredictionWithMatrixNew plus the finer-neighbour correction of
 * Sec. 6.1, boundaries by Eq. AdvectionOnBoundary) and the collision on the
 * leaves (Eq. AdaptiveCollision), and, for D2Q9 with an obstacle, the
 * penalisation of Sec. 7.2.2.
 *
 * Conventions shared by every entry point:
 *  - every function returns an mr_status and never aborts or throws;
 *  - errors are sticky per handle: once a call fails, later calls on the
 *    handle return the same status until mr_lbm_destroy();
 *  - work is ordered on the CUDA stream given at creation; calls that move
 *    data to host memory (on_device = 0) synchronise that stream, the others
 *    return as soon as the work is queued; device-side failures (capacity
 *    overflow, an inconsistent mesh, a non-finite value) are reported by the
 *    next call that synchronises (mr_lbm_synchronize, mr_lbm_stats, any
 *    copy to host);
 *  - the caller owns every pointer it passes; the handle owns all device
 *    memory it allocates (mr_lbm_create allocates, mr_lbm_destroy frees);
 *  - on_device = 1 means the pointer is device memory of the current device,
 *    on_device = 0 means host memory (pinned or pageable);
 *  - cells are indexed per level by integer coordinates k with
 *    0 <= k_a < roots[a] * 2^level (Sec. 2.1).  A key is the cell's Morton
 *    code at its own level prefixed by its root: key = root << (d*level) |
 *    interleave(k mod 2^level), interleave placing bit i of k_x at bit d*i,
 *    of k_y at bit d*i+1, root = (k_x >> level) + roots[0] * (k_y >> level).
 *    Leaves are returned sorted by (level, key).
 *  - dense arrays of one level are row-major with x fastest.
 */
#ifndef MR_LBM_H
#define MR_LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MR_OK = 0,
  MR_EINVAL = 1,      /* invalid argument or configuration */
  MR_ENOMEM = 2,      /* device or host allocation failed */
  MR_ECUDA = 3,       /* a CUDA runtime call failed */
  MR_ECAPACITY = 4,   /* more cells than the preallocated capacity */
  MR_ENOCONV = 5,     /* reserved: a bounded iteration did not converge */
  MR_ENONFINITE = 6,  /* a non-finite population appeared */
  MR_ESTATE = 7,      /* call not allowed in the current state (e.g. not initialised) */
  MR_EINTERNAL = 8    /* the mesh violated an invariant (a bug) */
} mr_status;

typedef enum {
  MR_D1Q2_ADVECTION = 0,     /* m^eq = (u, V u), V = phys[0] */
  MR_D1Q2_BURGERS = 1,       /* m^eq = (u, u^2/2) */
  MR_D1Q3_SHALLOW_WATER = 2, /* m^eq = (h, q, q^2/h + g h^2/2), g = phys[0] */
  MR_D2Q4x4_EULER = 3,       /* vectorial D2Q4^4 of Sec. 7.1.2, gamma = phys[0] */
  MR_D2Q9_NS = 4,            /* D2Q9 of Sec. 7.2.2 (orthogonal moments, Lallemand-Luo):
                                conserved (rho, q_x, q_y); s[0] relaxes the energy, energy
                                square and heat-flux moments, s[1] the two stress moments;
                                rho0 = phys[0], u0 = (phys[1], phys[2]) for
                                MR_BC_BOUNCE_BACK_VELOCITY and the obstacle; obstacle disc
                                centre (phys[3], phys[4]), radius phys[5].  Needs the
                                tensor-product prediction (cross_sign +1). */
  MR_D3Q6_ADVECTION = 5      /* D3Q6 of Sec. 7.3: eta = +-e_x, +-e_y, +-e_z, the printed M,
                                m^eq = (u, V_x u, V_y u, V_z u, 0, 0), V = phys[0..2];
                                s[0] = s1 (first moments), s[1] = s2 (the two second
                                moments); d = 3, keys are 3-way Morton codes with a root
                                prefix, max_level <= 10 */
} mr_scheme;

typedef enum {
  MR_BC_PERIODIC = 0,        /* both faces of an axis must be periodic */
  MR_BC_COPY = 1,            /* Eq. refBoundaryConditions, copy */
  MR_BC_BOUNCE_BACK = 2,     /* Eq. refBoundaryConditions, bounce back */
  MR_BC_ANTI_BOUNCE_BACK = 3, /* Eq. refBoundaryConditions, anti bounce back */
  MR_BC_BOUNCE_BACK_VELOCITY = 4 /* bounce back of a wall moving at u0 (Sec. 7.2.2, D2Q9 only):
                                    f^{h dagger} + f^{h,eq}(rho0, u0) - f^{h dagger,eq}(rho0, u0) */
} mr_bc;

/* Storage and arithmetic of the populations.  The details that decide the
 * mesh (Def. Details, Eq. Thresholding, the refinement rule) are evaluated
 * in FP64 in every form, on the stored values. */
typedef enum {
  MR_FP64 = 0,           /* plain: FP64 storage and arithmetic */
  MR_FP32 = 1,           /* FP32 storage, FP32 transport and collision */
  MR_FP32_FP16STORE = 2, /* FP16 storage of f - f^eq(mean initial state), FP32 arithmetic */
  MR_FP32_BF16STORE = 3  /* BF16 storage of f - f^eq(mean initial state), FP32 arithmetic */
} mr_precision;

typedef struct {
  int scheme;            /* mr_scheme */
  double lambda;         /* lattice velocity lambda = dx/dt, Eq. acousticscaling; > 0 */
  double s[16];          /* relaxation rates in [0, 2] of the non-conserved moments:
                            D1Q2: s[0]; D1Q3: s[0] (third moment);
                            D2Q4^4: s[i] = s_i^q, s[4+i] = s_i^xy, i = 0..3;
                            D2Q9: s[0] (energy, energy square, heat flux), s[1] (stress) */
  double phys[8];        /* scheme constants (see mr_scheme) */
  double xmin[3], xmax[3]; /* physical domain (used by the obstacle only) */
  int roots[3];          /* cells per axis at level 0 (1 for the unit square); MR_EINVAL
                            unless roots_x roots_y roots_z 2^(d max_level) <= 2^32 and
                            the cells of levels min_level..max_level number under 2^30 */
  int min_level, max_level; /* J_min and J; 2 <= J_min <= J <= 15 */
  double eps;            /* threshold epsilon >= 0, eps_j = 2^{d(j-J)} eps (Sec. 4.4) */
  int mu_bar;            /* regularity guess of the refinement rule, 0 .. 2s + 1 (Sec. 5.1) */
  int pred_s;            /* half-width s of the prediction operator, 1, 2 or 3 (Table 1; 0
                            reads as 1): (2s+1)^d stencils, grading of radius s, transport
                            windows of 2s cells (blocks of (4s+1)^2 cells for D2Q9).
                            mr_lbm_adjoint needs s = 1 (MR_EINVAL otherwise) */
  int bc[6];             /* mr_bc per face: -x, +x, -y, +y, -z, +z */
  int cross_sign;        /* +1: tensor-product prediction (default, also when 0);
                            -1: diagonal term with the sign printed in Sec. 4.1 */
  int precision;         /* mr_precision */
  long long leaf_capacity; /* maximum number of leaves; 0 = all finest cells */
  int obstacle;          /* 1: penalisation of Sec. 7.2.2 after each collision (D2Q9 only):
                            f <- phi f^eq(rho0, 0) + (1 - phi) f, phi = share of the leaf's
                            finest-cell centres inside the disc; xmin / xmax place the disc */
  int exact_collision;   /* 1: the "original adaptive" collision of Sec. 5.3 (the right-hand
                            side of Eq. sourceoferror): the post-transport data are
                            reconstructed on every finest cell, collided there and averaged
                            back onto each leaf, instead of colliding the leaf's averages
                            (Eq. AdaptiveCollision).  FP64 form only, single solvers only (not
                            in a batch, not with mr_lbm_adjoint); allocates a dense FP64
                            buffer of Q values per cell of levels min_level..max_level. */
} mr_lbm_config;

typedef struct mr_lbm* mr_lbm_t;

/* Create a solver for `cfg` on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream) on which all work is queued.
 * Allocates every device buffer up front (capacities from cfg); *out is NULL
 * on failure.  Does not initialise the field: call mr_lbm_init or
 * mr_lbm_set_leaves next. */
mr_status mr_lbm_create(const mr_lbm_config* cfg, void* cuda_stream, mr_lbm_t* out);

/* Release all memory of the handle.  Accepts NULL. */
mr_status mr_lbm_destroy(mr_lbm_t h);

/* Algorithm 1 initialisation: the full finest mesh Lambda(0) with
 * f = M^{-1} m^eq of the given conserved moments.  `conserved` is SoA
 * [ncons][N_J] of doubles, N_J = prod_a roots[a] 2^J cells of level J,
 * row-major (x fastest); ncons = 1 (D1Q2), 2 (D1Q3), 4 (D2Q4^4:
 * rho, rho u, rho v, E), 3 (D2Q9: rho, q_x, q_y). */
mr_status mr_lbm_init(mr_lbm_t h, const double* conserved, int on_device);

/* `nsteps` iterations of the loop of Algorithm 1: adapt the mesh from the
 * details of the stored post-collision field, move the data to the new
 * leaves, stream every leaf (Eq. AdaptiveAdvectionPhase) and collide it
 * (Eq. AdaptiveCollision).  Asynchronous. */
mr_status mr_lbm_step(mr_lbm_t h, int nsteps);

/* Mesh adaptation and data transfer only (first two lines of the loop of
 * Algorithm 1), without transport and collision.  Asynchronous. */
mr_status mr_lbm_adapt(mr_lbm_t h);

/* Conserved moments of the reconstructed field on the uniform level `level`
 * (J_min <= level <= J): the average of the leaves for cells covered by finer
 * leaves, the recursive prediction (reconstruction operator, Sec. 4.4) for
 * cells inside coarser leaves.  `out` is SoA [ncons][N_level], row-major. */
mr_status mr_lbm_project(mr_lbm_t h, int level, double* out, int on_device);

/* Same result as mr_lbm_project, for callers that must not allocate memory
 * during the call (the paper has no counterpart: this is a deployment aid).
 * mr_lbm_project allocates its two dense level buffers on first use; a caller
 * whose device memory belongs to another allocator with a fixed budget (a
 * framework's caching allocator, a memory pool), or a serving loop that
 * cannot afford the device-wide synchronisation an allocation may cause,
 * cannot let that happen.  This variant calls no cudaMalloc, cudaFree or
 * allocating library routine: its level buffers live in one file-scope
 * device array of 2^21 doubles (16 MiB) that each GPU loading the library
 * holds until the process exits.  Limit: ncons * N_level <= 2^20 (e.g. the
 * D2Q4^4 Euler scheme up to level 9); larger levels return MR_ECAPACITY
 * without touching the handle, which stays usable.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make it before any stream capture.  All calls on a
 * device share the array and its leftover contents (nothing in it has to
 * start at zero); calls whose GPU work overlaps race on it, so serialise
 * them.  Arguments, layout and synchronisation as in mr_lbm_project. */
mr_status mr_lbm_project_noalloc(mr_lbm_t h, int level, double* out, int on_device);

/* Copy the leaves out, sorted by (level, key).  Call with keys = levels =
 * f = NULL to query the count in *n_inout; otherwise *n_inout is the capacity
 * of the buffers on entry and the number written on return (MR_EINVAL if too
 * small).  f is SoA [Q][n] of doubles, Q = populations per cell (2, 3, 16). */
mr_status mr_lbm_get_leaves(mr_lbm_t h, long long* n_inout, unsigned long long* keys,
                            signed char* levels, double* f, int on_device);

/* Replace the state by the given leaves (any order), which must partition the
 * domain and form a graded tree (every state produced by mr_lbm_step does).
 * keys/levels as in mr_lbm_get_leaves, f SoA [Q][n].  Duplicate or
 * overlapping leaves, or leaves that do not cover the domain, give
 * MR_EINVAL at the next synchronising call.  With host buffers (on_device =
 * 0) the call returns once it has read them (pinned buffers are copied
 * asynchronously, the populations on a second stream of the handle, while
 * the mesh is built); the build and the gather of the values may still be
 * running on the handle's stream, and their device-side errors come back at
 * the next synchronising call. */
mr_status mr_lbm_set_leaves(mr_lbm_t h, long long n, const unsigned long long* keys,
                            const signed char* levels, const double* f, int on_device);

/* Mesh statistics (synchronises): leaves per level (array of J+1 entries,
 * may be NULL), MeshOR = #leaves / #finest cells and MemOR = #cells of the
 * complete tree / #cells of all levels J_min..J (Sec. 7.1.3). */
mr_status mr_lbm_stats(mr_lbm_t h, long long* leaves_per_level, double* mesh_or, double* mem_or);

/* Sum over all steps since creation of the number of leaves updated (device
 * counter, synchronises), and the number of steps. */
mr_status mr_lbm_counters(mr_lbm_t h, long long* leaf_updates, long long* steps);

/* Number of kernels the handle has launched since creation (host counter). */
long long mr_lbm_launch_count(mr_lbm_t h);

/* Time every launch of one kernel group with a pair of CUDA events on the
 * handle's stream: on = 1 transport+collision, 2 details, 3 projection,
 * 4 ghost / new-leaf prediction, 5 mesh adaptation and compaction,
 * 6 data transfer; 0 disables.  mr_lbm_profile_read synchronises and returns
 * the total milliseconds and the number of timed launches since the last
 * mr_lbm_profile_enable. */
mr_status mr_lbm_profile_enable(mr_lbm_t h, int on);
mr_status mr_lbm_profile_read(mr_lbm_t h, double* total_ms, long long* launches);

/* Wait for the handle's stream and report any deferred device-side error. */
mr_status mr_lbm_synchronize(mr_lbm_t h);

/* Human-readable name of a status. */
const char* mr_lbm_strerror(mr_status s);

/* Host-only introspection (needs no GPU): the flattened weights of
 * Eq. PredictionWithMatrixNew used by the transport for a leaf of level
 * `level` at position k along an axis of n_level = roots << level cells
 * (periodic or not) when the finest level is `max_level`.  out[0..4] are the
 * weights of f_{level,k+delta}, delta = -2..2, in (incoming - outgoing) for
 * the velocity +1 along the axis, out[5..9] for the velocity -1 (the part
 * entering through a non-periodic boundary is left out). */
mr_status mr_lbm_flattened_weights(int roots, int level, int max_level, int periodic, int k,
                                   double* out);

/* Host-only: the same weights for the prediction of half-width s = 1, 2, 3
 * (Table 1; Sec. 4.1) over the window delta = -half_width..half_width:
 * out[0 .. 2w] for the velocity +1, out[2w+1 .. 4w+1] for -1 (w =
 * half_width; 4w + 2 doubles), max_level - level <= 12.  MR_EINVAL if a cell
 * outside the window carries a nonzero weight (the window is too narrow for
 * this s and gap) or an argument is out of range.  s = 1 with half_width 2
 * gives the weights of mr_lbm_flattened_weights. */
mr_status mr_lbm_flattened_weights_s(int s, int half_width, int roots, int level, int max_level,
                                     int periodic, int k, double* out);

/* ------------------------------------------------------------------ adjoint
 * Gradients of a functional of the trajectory through the time steps with
 * the mesh of every step frozen (the adaptation decisions of the forward
 * pass are replayed, not differentiated).  The transfer, ghost prediction,
 * projection and transport are linear for a given mesh; their adjoints are
 * transposed scatters, and the collision (and obstacle) Jacobians come from
 * the scheme's own code on dual numbers.  Memory: a checkpoint of the leaves
 * every `checkpoint_every` steps; the backward pass replays one segment at
 * a time from its checkpoint, recording its meshes and pre-collision states.
 *
 * Functionals, with E(x) = sum over the leaves of |cell| |q|^2 / (2 rho)
 * (conserved moments rho = u_0, q = (u_1, u_2); 1/2 u_0^2 for a scheme with
 * one conserved moment; |cell| = dx^d 2^{d (J - level)}):
 *   MR_FUNCTIONAL_KE_SUM:   J = sum_{n = 1..nsteps} E(x_n),
 *   MR_FUNCTIONAL_KE_FINAL: J = E(x_nsteps). */
typedef enum { MR_FUNCTIONAL_KE_SUM = 1, MR_FUNCTIONAL_KE_FINAL = 2 } mr_functional;

/* Initialise from `conserved0` (layout and `on_device` as mr_lbm_init), run
 * `nsteps` steps, and return J (*J_out, host), dJ/d conserved0
 * (grad_conserved0, same layout and memory kind as conserved0) and dJ/d s
 * (grad_s[16], host, for the 16 relaxation-rate slots of the config).  With
 * both gradient pointers NULL only J is computed.  FP64 form only
 * (MR_EINVAL otherwise); a batch member returns MR_ESTATE.  On return the
 * handle holds the state after nsteps steps.  Synchronises. */
mr_status mr_lbm_adjoint(mr_lbm_t h, const double* conserved0, int on_device, int nsteps, int checkpoint_every,
                         int functional, double* J_out, double* grad_conserved0, double* grad_s);

/* ------------------------------------------------------------------ batches
 * Many independent solvers (any mix of schemes, levels, thresholds and
 * forms) stepped together: every kernel of a time step runs once for all
 * instances of the same scheme and storage form, whose uneven leaf counts
 * are spread over the whole GPU, and the step is replayed from a CUDA graph
 * in which instances of different schemes or forms are concurrent branches.
 * The batch owns its instances; mr_lbm_batch_instance lends one as an
 * ordinary handle for mr_lbm_init, mr_lbm_set_leaves, mr_lbm_get_leaves,
 * mr_lbm_project, mr_lbm_stats and mr_lbm_counters.  mr_lbm_step,
 * mr_lbm_adapt and mr_lbm_destroy refuse a lent handle with MR_ESTATE (the
 * instances share one mesh parity). */
typedef struct mr_lbm_batch* mr_lbm_batch_t;

/* Create n solvers from cfgs[0..n-1] on the current device, all queued on
 * `cuda_stream`.  Fails with the first failing instance's status. */
mr_status mr_lbm_batch_create(const mr_lbm_config* cfgs, int n, void* cuda_stream, mr_lbm_batch_t* out);
/* Borrow instance i (0 <= i < n, in the order of cfgs). */
mr_status mr_lbm_batch_instance(mr_lbm_batch_t b, int i, mr_lbm_t* out);
/* `nsteps` steps of Algorithm 1 for every instance (all must be
 * initialised: MR_ESTATE otherwise).  Asynchronous. */
mr_status mr_lbm_batch_step(mr_lbm_batch_t b, int nsteps);
/* Wait and report the first deferred device-side error of any instance. */
mr_status mr_lbm_batch_synchronize(mr_lbm_batch_t b);
/* Sum of the instances' leaf updates; the number of steps taken. */
mr_status mr_lbm_batch_counters(mr_lbm_batch_t b, long long* leaf_updates, long long* steps);
/* Kernel launches queued by the batch's steps. */
long long mr_lbm_batch_launch_count(mr_lbm_batch_t b);
/* Event timing of one kernel group of the batched steps (groups as for
 * mr_lbm_profile_enable). */
mr_status mr_lbm_batch_profile_enable(mr_lbm_batch_t b, int group);
mr_status mr_lbm_batch_profile_read(mr_lbm_batch_t b, double* total_ms, long long* launches);

/* Launch schedules of the batched form (the paper has no counterpart: this
 * is how the batch maps onto the GPU).  The instances of one half-width,
 * scheme and storage form make a part, stepped by shared grid-stride
 * launches; a part's schedule gives, for each of its MR_LBM_NPHASE phases,
 * the blocks per SM its tiled kernels may use (the grid is capped at that
 * many blocks per SM; blocks stride over the tiles).  Phases, in order:
 * projection, details, mesh flags and grading, compaction, data transfer,
 * ghost / new-leaf prediction, transport + collision.  Defaults
 * {8, 8, 4, 8, 8, 8, 8}.  mr_lbm_batch_parts gives the number of parts;
 * get / set read and write one part's schedule (values 1..64, else
 * MR_EINVAL; set synchronises the batch's stream). */
#define MR_LBM_NPHASE 7
mr_status mr_lbm_batch_parts(mr_lbm_batch_t b, int* nparts);
mr_status mr_lbm_batch_get_schedule(mr_lbm_batch_t b, int part, int* bps /* [MR_LBM_NPHASE] */);
mr_status mr_lbm_batch_set_schedule(mr_lbm_batch_t b, int part, const int* bps /* [MR_LBM_NPHASE] */);

/* Autotuner of the schedules: coordinate descent over each part and phase,
 * candidates 1, 2, 4, 8, 16, 32 blocks per SM, each candidate timed (CUDA
 * events on the batch's stream, graph replay) over `trial_steps` batched
 * steps (1..1000) from the same state, a change kept only if the step gets
 * more than 1 % faster.  Every instance is snapshotted first (device
 * buffers the tuner allocates and frees) and put back afterwards, with its
 * counters: the batch leaves the call in the state it entered it.
 * *ms_fixed / *ms_tuned (may be NULL): time per step of the schedule on
 * entry and of the chosen one.  The result is cached for the batch's
 * signature (per part: half-width, scheme, form, instance count and the
 * power of two of the mean finest-cell count): later batches of the same
 * signature in the process start from it, and so do those of later
 * processes when the environment variable MR_LBM_TUNE_CACHE names a file
 * (one line per tuning is appended).  Synchronises; minutes for large
 * batches (7 phases x 5 candidates x parts trials). */
mr_status mr_lbm_batch_autotune(mr_lbm_batch_t b, int trial_steps, double* ms_fixed, double* ms_tuned);

/* Release the batch and all its instances.  Accepts NULL. */
mr_status mr_lbm_batch_destroy(mr_lbm_batch_t b);

#ifdef __cplusplus
}
#endif
#endif /* MR_LBM_H */
