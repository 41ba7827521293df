/*
 * p3t.h -- C ABI of libp3t, the GB300 (sm_103a) soft step of the
 * particle-particle particle-tree (P3T) planetary N-body integrator with
 * individual cut-off radii (Ishigaki, Kominami, Makino, Fujimoto & Iwasawa
 * 2021, PASJ 73, 660: "GPLUM").
 *
 * One soft step (Sec. 2.2, procedure steps 3-8; Eq. HamiltonSol) is
 *
 *   p3t_kick        v += a_soft dt/2
 *   p3t_hard_step   Hermite-4 for every neighbour cluster, Kepler drift for
 *                   isolated particles, over dt
 *   p3t_build_tree  Morton keys, sort, octree with monopole + quadrupole
 *   p3t_soft_force  tree walk with the changeover function -> a_soft,
 *                   neighbour candidates, interaction counts
 *   p3t_neighbours  neighbour lists (CSR) and neighbour clusters
 *   p3t_kick        v += a_soft dt/2
 *
 * Conventions shared by every entry point
 *  - Particles are structure-of-arrays of FP64 in the CALLER's order; every
 *    output is in the caller's order too (the library sorts internally and
 *    scatters back).  Particle indices are int32 (n < 2^31), CSR offsets int64.
 *  - Unless stated otherwise a pointer argument is a DEVICE pointer on the
 *    context's device, owned by the caller, and must stay valid until the
 *    work queued on the stream has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every compute entry point only enqueues work: it neither
 *    allocates (once p3t_reserve has sized the context) nor synchronises, so
 *    a sequence of calls can be captured into a CUDA graph.
 *  - Return value: 0 or a negative P3T_ERR_* code for errors detected on the
 *    host (bad arguments, failed launches).  Errors found while the kernels
 *    run (a full buffer, a Hermite step below dt/2^40) are recorded on the
 *    device, are sticky, and are read and cleared by p3t_status.
 *  - Kernels never trap and never spin without a bound.
 *  - Units are the caller's; the paper uses G = M_* = 1, au, yr/2pi (Sec. 3.1).
 */
#ifndef P3T_H
#define P3T_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define P3T_OK 0
#define P3T_ERR_INVALID (-1)       /* bad argument, parameter or call order   */
#define P3T_ERR_CUDA (-2)          /* a CUDA runtime call or launch failed     */
#define P3T_ERR_CAPACITY (-3)      /* an output or internal buffer is too small;
                                      p3t_status reports the size needed      */
#define P3T_ERR_DT_UNDERFLOW (-4)  /* a Hermite step fell below dt / 2^40      */
#define P3T_ERR_TIMEOUT (-5)       /* a bounded device loop gave up            */

#define P3T_FP64 0   /* every step in FP64                                     */
#define P3T_MIXED 1  /* pair arithmetic of the soft force in FP32 on relative
                        coordinates of FP64 accuracy (float-float split),
                        FP32 pair terms folded into float-float accumulators;
                        FP64 state, tree, neighbour search, Hermite, Kepler   */

/* cut-off radius schemes (Sec. 2.1.1-2.1.3), p3t_params.cutoff_mode */
#define P3T_CUT_HILL_VRAN 0  /* Hill radius and random velocity (Eq. routi2)   */
#define P3T_CUT_HILL 1       /* Hill radius only (Eq. routi)                   */
#define P3T_CUT_SHARED 2     /* one shared radius (Eq. rout1)                  */

/* ---- method parameters (defaults: the paper's values, Sec. 3.1) --------- */
typedef struct {
  double G;        /* gravitational constant                                  */
  double m_star;   /* mass of the central star M_*                            */
  double dt_soft;  /* soft step Delta t (Eq. HamiltonSol); used by the cut-off
                      and neighbour rules (Eqs. routi2, rsearch, rsearch1)     */
  double gamma;    /* r_in / r_out of the changeover, 0 < gamma < 1 (Sec. 2.1.1) */
  double rcut0;    /* R~cut,0: Hill-radius factor (Eq. routi2)                 */
  double rcut1;    /* R~cut,1: random-velocity factor (Eq. routi2), paper: 8   */
  double rs0, rs1; /* R~search,0 / R~search,1 (Eq. rsearch), paper: 1.1, 6     */
  double rs2, rs3; /* R~search,2 / R~search,3 (Eq. rsearch1), paper: 2, 2      */
  double theta;    /* Barnes-Hut opening angle (Sec. 3.1: 0.1 or 0.5); 0 =
                      direct summation                                        */
  double eta;      /* Hermite accuracy parameter (Sec. 3.1: 0.01)             */
  double eta0;     /* Hermite first-step parameter (Sec. 3.1: 0.1 eta)        */
  double f_radius; /* collision radius factor f (Sec. 2.4.1: two particles
                      collide when r_ij < f (R_p,i + R_p,j); the paper uses
                      1); 0 = no collisions.  Collisions also need r_phys. */
  int32_t leaf_size; /* max particles per leaf = per target group, 1..32      */
  int32_t precision; /* P3T_FP64 or P3T_MIXED                                  */
  int32_t vran_bins; /* radial bins for v_ran; 0 = clamp(N/1000, 1, 1024)      */
  int32_t group_size;/* target groups of the walk: the highest tree nodes holding
                        <= group_size particles (0: every leaf is a group);
                        0..64                                                 */
  int32_t cutoff_mode;/* P3T_CUT_HILL_VRAN (default): r_out,i = max(R~cut,0
                        r_Hill,i, R~cut,1 v_ran,i dt) (Eq. routi2);
                        P3T_CUT_HILL: R~cut,0 r_Hill,i (Eq. routi);
                        P3T_CUT_SHARED: every particle gets the largest
                        Eq. routi radius and the largest search radius
                        (Eq. rout1, the "shared cut-off")                     */
} p3t_params;

/* ---- particles ---------------------------------------------------------- */
typedef struct {
  int64_t n;                       /* number of particles, 0 <= n < 2^31     */
  double *x, *y, *z;               /* positions, n each                      */
  double *vx, *vy, *vz;            /* velocities, n each                     */
  double *m;                       /* masses, n, > 0                         */
  double *r_out, *r_search;        /* cut-off and search radii, n each; written
                                      by p3t_cutoffs (or p3t_build_tree with
                                      update_cutoffs = 1), read by the rest   */
  double *r_phys;                  /* physical radii R_p, n, or NULL (no
                                      collisions); read by p3t_hard_step,
                                      written by p3t_merge                    */
} p3t_particles;

/* ---- neighbour clusters: library-owned device views ---------------------- */
typedef struct {
  const int32_t *label;   /* n: smallest particle index of the particle's
                             neighbour cluster (Sec. 2.3, steps i-iii)        */
  const int32_t *singles; /* counts[0]: isolated particles, ascending          */
  const int64_t *cl_off;  /* counts[1] + 1: offsets of clusters of >= 2       */
  const int32_t *cl_mem;  /* counts[2]: members, clusters ordered by label,
                             members ascending                                 */
  const int64_t *counts;  /* device int64[4]: n_single, n_clusters, n_members,
                             size of the largest cluster                       */
} p3t_clusters;

typedef struct p3t_ctx p3t_ctx;

/* Creates a context on CUDA device `device` with parameters *p (copied).
 * The context owns the tree, the sorted copies, all scratch and the cluster
 * views.  Returns P3T_ERR_INVALID for out-of-range parameters. */
int p3t_create(p3t_ctx **ctx, const p3t_params *p, int device);

/* Frees everything the context owns (synchronises its device first). */
void p3t_destroy(p3t_ctx *ctx);

/* Replaces the parameters (host call; takes effect for work enqueued after).
 * A change of leaf_size, group_size or precision drops the tree (its sorted
 * copies and moments are those of one precision): p3t_build_tree again
 * before the next p3t_soft_force or p3t_neighbours. */
int p3t_set_params(p3t_ctx *ctx, const p3t_params *p);

/* Sizes every internal buffer for up to n particles (allocates, so call it
 * before any graph capture).  Compute calls with a larger n grow the context
 * themselves, which allocates and is then not capturable. */
int p3t_reserve(p3t_ctx *ctx, int64_t n);

/* Batched ensemble: the particles of the following calls form nseg
 * independent systems (disks) stored one after another, system d being
 * [seg_off[d], seg_off[d + 1]) (host array of nseg + 1 offsets, seg_off[0]
 * = 0, strictly increasing, copied; the sum below 2^31).  With nseg > 1
 * every stage keeps the systems apart exactly as if each had a context of
 * its own, and each system gets the same bits as it would alone: the cut-off
 * radii use each system's own radial bins (Sec. 2.1.3; the bins of all
 * systems together at most 4096, else P3T_ERR_INVALID from the cut-off
 * calls), each system gets its own root cube, key grid and octree (one tree
 * per system in the shared node arrays; the root of system d is node d), the
 * walk of a target group starts at its system's root, so no force,
 * neighbour or cluster links two systems (Sec. 2.3: clusters are
 * independent).  One group size, leaf size and parameter set for all.  The
 * particle count of later calls must equal seg_off[nseg] (else
 * P3T_ERR_INVALID); p3t_energy, p3t_merge, p3t_soft_force_direct and
 * p3t_soft_force_vjp return P3T_ERR_INVALID while nseg > 1.  nseg = 1
 * restores the single system.  Returns P3T_ERR_INVALID for bad offsets or
 * nseg outside [1, 4096] (the context keeps its previous segments) and
 * P3T_ERR_CUDA when an allocation fails (the context is then a single
 * system).  Synchronises the device and allocates: call it before any graph
 * capture; it drops the context's tree. */
int p3t_set_segments(p3t_ctx *ctx, int64_t nseg, const int64_t *seg_off);

/* Cut-off and search radii, Eq. routi2 and Eq. rsearch:
 *   r_out,i    = max(R~cut,0 r_Hill,i, R~cut,1 v_ran,i dt_soft),
 *   r_Hill,i   = (m_i / 3M_*)^(1/3) a_i, a_i the osculating semi-major axis
 *                (a_i = |x_i| for an unbound orbit),
 *   r_search,i = R~s,0 r_out,i + R~s,1 v_ran,i dt_soft,
 * v_ran,i = rms of |v - sqrt(G M_* / |x|) phi_hat| over the particle's radial
 * bin (bins uniform in ln of the cylindrical radius).  Writes p->r_out and
 * p->r_search. */
int p3t_cutoffs(p3t_ctx *ctx, p3t_particles *p, void *stream);

/* Cut-off and search radii without a context and without any allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- an application that owns all device memory through its own
 * pool and forbids other allocations (a plugin host, a framework with a fixed
 * memory budget), or a latency-critical loop where the synchronisation
 * cudaMalloc and cudaFree may imply would stall other work.  Such callers
 * cannot create a context (p3t_create allocates) but can call this.
 *  - Same results as p3t_cutoffs for the same parameters and particles to a
 *    few ulp: the radial-bin sums of |u|^2 are exact 128-bit fixed-point sums
 *    of terms cut to multiples of 2^-88 (|u|^2 below 2^40), so every run gives
 *    the same bits, but not p3t_cutoffs' FP64 sums.
 *  - Runs on the CURRENT CUDA device; all particle pointers must be on it.
 *    p and *p are host memory; the arrays they point to are device memory
 *    owned by the caller (inputs x..m are read, r_out and r_search written).
 *  - Scratch: a fixed 98,320-byte array in device memory that every GPU
 *    loading the library holds until the process exits; at most 4096 radial
 *    bins (prm->vran_bins > 4096 returns P3T_ERR_INVALID; the automatic choice
 *    is at most 1024).  Each call clears what it uses before use.
 *  - The first call on a device looks up the scratch address on that device
 *    (a host-side runtime query); make that first call before any stream
 *    capture.
 *  - Every call shares the scratch: calls that overlap on the GPU (e.g. on
 *    two streams with no ordering between them) race and must be avoided.
 *  - cutoff_mode P3T_CUT_HILL_VRAN or P3T_CUT_HILL only; the shared radius
 *    (a maximum over all particles) returns P3T_ERR_INVALID.
 *  - Returns 0, P3T_ERR_INVALID (bad arguments, too many bins, shared mode) or
 *    P3T_ERR_CUDA (the lookup or a launch failed). */
int p3t_cutoffs_noalloc(const p3t_params *prm, p3t_particles *p, void *stream);

/* Morton keys on the 21-bit grid of the cubic bounding box,
 * stable sort by (key, index), octree (split while > leaf_size particles and
 * level < 21), per node mass, centre of mass, traceless quadrupole
 * Q_ab = sum m (3 d_a d_b - d^2 delta_ab), quantised tight box and search
 * reach.  The tree stays in the context for p3t_soft_force.  With
 * update_cutoffs = 1, p3t_cutoffs runs first.  (Sec. 2.1.2: the paper's soft
 * force uses a Barnes-Hut tree.) */
int p3t_build_tree(p3t_ctx *ctx, p3t_particles *p, int update_cutoffs,
                   void *stream);

/* Soft acceleration, Eq. softforce:
 *   a_i = -sum_j G m_j K(r_ij / r_out,ij) r_ij / r_ij^3,
 *   r_out,ij = max(r_out,i, r_out,j) (Eq. rout2), K the changeover of
 *   Sec. 2.1.1 (zero below gamma, one above 1),
 * by a tree walk per target group (a node holding <= group_size particles
 * whose parent holds more, or a leaf): accepted nodes add monopole +
 * quadrupole, opened leaves add the changeover pair terms.  A node is opened when the
 * Barnes-Hut test fails or it lies within the search reach, so all pairs with
 * r_ij < max(r_search,i, r_search,j) are evaluated as pairs and recorded as
 * neighbour candidates for p3t_neighbours.  p must be the particles the tree
 * was built from.  ax, ay, az: n doubles each (caller order, overwritten).
 * counts: NULL or a device uint64[2] overwritten with the numbers of
 * particle-particle and particle-node terms evaluated. */
int p3t_soft_force(p3t_ctx *ctx, const p3t_particles *p, double *ax, double *ay,
                   double *az, uint64_t *counts, void *stream);

/* Neighbour lists and clusters, Sec. 2.3:
 * a candidate j of i stays a neighbour iff r_ij < r_search,ij and either its
 * closest approach under linear motion over [0, dt_soft] (Eq. rsearch1 with
 * t_min) is at most R~s,2 r_out,ij, or v_ij < R~s,3 a_ij dt_soft / 2 with
 * a_ij = G (m_i + m_j) / r_ij^2; all tests in FP64.  Lists are symmetric.
 * nb_off: device int64[n+1], nb_idx: device int32[nb_cap], rows sorted by j.
 * If more than nb_cap entries are needed, nb_off is still complete, nb_idx
 * holds the first nb_cap, no clusters are formed and P3T_ERR_CAPACITY is
 * recorded with the size needed.  Clusters are the connected components of
 * the neighbour graph labelled by their smallest index (the fixed point of
 * the paper's min-label propagation).  *out receives library-owned views,
 * valid until the next p3t_neighbours call on this context.  Must follow
 * p3t_soft_force on the same particles. */
int p3t_neighbours(p3t_ctx *ctx, const p3t_particles *p, int64_t *nb_off,
                   int32_t *nb_idx, int64_t nb_cap, p3t_clusters *out,
                   void *stream);

/* Hard part over [0, dt] (procedure step 5, Eq. hardforce):
 * every cluster of >= 2 members is integrated with the fourth-order Hermite
 * predictor-corrector and block individual time steps (dt / 2^k, k <= 40;
 * Aarseth step with eta, first step eta0 |a|/|j|), under the star and the
 * (1 - K) part of the pair forces; every isolated particle is advanced on its
 * Kepler orbit about M_* (universal variables, Newton-Raphson).  Positions and
 * velocities of p are updated in place.  cl: views from p3t_neighbours or
 * caller-built device arrays of the same layout.  n_steps: NULL or a device
 * uint64 overwritten with the number of Hermite particle-steps.
 * Perfect accretion (Sec. 2.4.1), with f_radius > 0 and p->r_phys set: at
 * every force evaluation of the block steps a member that touches another
 * (r_ij < f (R_p,i + R_p,j)) joins it in a composite that moves as one body
 * (centre-of-mass position and velocity, mass-weighted mean hard force, a
 * fresh eta0 step); the members stay separate particles, recorded in the
 * context for the second p3t_kick and p3t_merge, which must follow before
 * the next p3t_hard_step. */
int p3t_hard_step(p3t_ctx *ctx, p3t_particles *p, const p3t_clusters *cl,
                  double dt, uint64_t *n_steps, void *stream);

/* The Kepler drift of p3t_hard_step applied to
 * all particles of p by dt (mu = G M_*), with no cluster integrated: the
 * drift of a rollout whose particles are all treated as isolated (the
 * adjoint's forward map).  Positions and velocities updated in place;
 * a drift whose Newton iteration does not converge is reported as
 * P3T_ERR_TIMEOUT by p3t_status. */
int p3t_kepler_drift(p3t_ctx *ctx, p3t_particles *p, double dt, void *stream);

/* Soft kick (procedure steps 3 and 8): v += a * h, h usually
 * dt_soft / 2.  ax, ay, az: n doubles each, caller order.  Members of a
 * composite formed by the last p3t_hard_step (f_radius > 0) are kicked with
 * the composite's mass-weighted mean acceleration (Sec. 2.4.1). */
int p3t_kick(p3t_ctx *ctx, p3t_particles *p, const double *ax, const double *ay,
             const double *az, double h, void *stream);

/* Procedure step 9 for collisions (Sec. 2.4.1, beyond the soft step):
 * replaces every composite formed by the last p3t_hard_step by one particle
 * at the lowest index of its members, with mass sum m_l, physical radius
 * (sum R_l^3)^(1/3) (one density for all bodies) and the members' common
 * position and velocity (call after the second p3t_kick).  The other members
 * are removed from the ten particle arrays, the survivors keep their order,
 * and p->n is set to the new count.  new_index: NULL or device int32[old n],
 * each particle's new index or -1.  e_disp: NULL or host double[2], the
 * energy dissipated since the last merge {in the hard part (Eq. edisphard,
 * changeover functions replaced by unity, the cluster standing for the
 * neighbour lists), by the averaged kick (E_disp,Soft)}.  n_merged: NULL or
 * host, number of particles removed.  Synchronises `stream`; not capturable.
 * After a merge the caller recomputes the cut-off radii, the tree, the soft
 * force and the neighbours (procedure step 9). */
int p3t_merge(p3t_ctx *ctx, p3t_particles *p, int32_t *new_index, double *e_disp,
              int64_t *n_merged, void *stream);

/* Whether the last p3t_hard_step formed composites that p3t_merge has not
 * yet merged (Sec. 2.4.1): *n_clusters (host) receives the number of
 * clusters in which composites formed, 0 when the step had no collision (or
 * f_radius = 0).  Synchronises `stream`;
 * not capturable.  A caller that learns of pending merges right after the
 * hard step may leave out the neighbour lists of the force that precedes
 * the merge (procedure step 7): the recomputation after the merge
 * (procedure step 9) replaces them before any hard step reads them. */
int p3t_collisions_pending(p3t_ctx *ctx, int64_t *n_clusters, void *stream);

/* The same count without synchronising the stream (Sec. 2.4.1, procedure
 * steps 7 and 9).  p3t_collisions_pending_async queues on `stream` a copy of
 * the count into host memory that the context owns and returns at once; work
 * queued after it (the tree and the soft force, which do not depend on it)
 * runs on.  p3t_collisions_pending_wait blocks until that copy alone has
 * landed and stores the count in *n_clusters (host).  One wait per queued
 * copy: P3T_ERR_INVALID when none is queued (the wait consumes it), and a
 * second _async before the wait replaces the first.  Neither is capturable
 * into a graph whose replay the caller does not wait for. */
int p3t_collisions_pending_async(p3t_ctx *ctx, void *stream);
int p3t_collisions_pending_wait(p3t_ctx *ctx, int64_t *n_clusters);

/* The soft force at theta = 0 (and the forward force of the adjoint) -- the
 * soft force of Eq. softforce summed directly over all pairs, which is what
 * the tree walk gives at theta = 0:
 *   a_i = -G sum_{j != i} m_j K(r_ij / r_out,ij) r_ij / r_ij^3,
 * r_out,ij = max(r_out,i, r_out,j); the central star is not included (it is
 * in the hard part's Kepler drift).  ax, ay, az: device, n each, caller
 * order, OVERWRITTEN.  P3T_FP64: FP64 arithmetic; P3T_MIXED: float-float
 * positions, FP32 pair terms, float-float sums.  Deterministic (fixed
 * summation order).  O(n^2): for small n and for the adjoint. */
int p3t_soft_force_direct(p3t_ctx *ctx, const p3t_particles *p, double *ax, double *ay,
                          double *az, void *stream);

/* Adjoint of the soft kick-drift-kick (the paper has no counterpart:
 * a gradient of a trajectory with respect to its initial state) -- the
 * vector-Jacobian product of the soft force of Eq. softforce with the cut-off
 * radii held fixed, taken for the direct sum over all pairs (the force the
 * tree approximates; exact at theta = 0):
 *   g_k += h G sum_j J(r_kj) (m_k lam_j - m_j lam_k),
 *   gm_k += h G sum_j phi_kj lam_j . r_kj,
 * J = phi I + psi r r^T the derivative of F(r) = K(|r|/r_out) r / |r|^3,
 * phi = K / r^3, psi = K'(y) / (r_out r^4) - 3 K / r^5.  That is, with
 * lam the adjoint of the velocity after a kick v += h a, the contributions
 * of that kick to the adjoints of the positions (gx, gy, gz) and masses (gm),
 * ADDED to what the arrays hold.  lx, ly, lz, gx..gm: device, n each, caller
 * order.  Arithmetic as p3t_soft_force_direct (FP64, or FP32 pair terms with
 * P3T_MIXED); deterministic.  O(n^2). */
int p3t_soft_force_vjp(p3t_ctx *ctx, const p3t_particles *p, double h, const double *lx,
                       const double *ly, const double *lz, double *gx, double *gy, double *gz,
                       double *gm, void *stream);

/* Adjoint of the tree soft force (the paper has no counterpart): the
 * vector-Jacobian product of Eq. softforce as p3t_soft_force evaluates it
 * with the tree, the interaction lists (which nodes are accepted and which
 * leaves are opened for each target group) and the cut-off radii held fixed:
 * a second walk of the context's tree meets the lists of the forward walk.
 * With L = sum_i lam_i . a_i, ADDS h dL/dx_i to (gx, gy, gz) and h dL/dm_i
 * to gm; node terms reach the particles through the node's mass, centre of
 * mass and quadrupole.  Requires a P3T_FP64 context whose tree was built
 * from p (p3t_build_tree; else P3T_ERR_INVALID).  lx, ly, lz, gx..gm:
 * device, n each, caller order.  FP64 arithmetic; contributions reach the
 * sums through atomic additions, so the last bits can differ between runs.
 * The first call allocates a per-node buffer (call it before any capture). */
int p3t_soft_force_vjp_tree(p3t_ctx *ctx, const p3t_particles *p, double h, const double *lx,
                            const double *ly, const double *lz, double *gx, double *gy,
                            double *gz, double *gm, void *stream);

/* Adjoint of the hard part of a soft step (the paper has no counterpart;
 * procedure step 5 with the neighbour clusters and the block schedule held
 * fixed): on entry lx..lvz hold the adjoint of the state after
 * p3t_hard_step(ctx, p, cl, dt), on return the adjoint of the state p holds
 * (the state BEFORE the hard step), and h-independent mass terms dL/dm of
 * the cluster members are ADDED to gm.  Isolated particles: the Kepler
 * drift's adjoint (as p3t_kepler_vjp); members of clusters of >= 2: the
 * derivative of the Hermite-4 block-step integration through forward-mode
 * tangents (one per member state component and mass), each integration in
 * plain FP64 with its step decisions taken on the values, so with the
 * schedule fixed.  Clusters of more than 16 members are not handled
 * (P3T_ERR_CAPACITY recorded).  No collisions (f_radius must be 0, else
 * P3T_ERR_INVALID).  cl: the clusters the forward hard step used.  Device
 * arrays, n each, caller order.  The first call allocates a buffer (call it
 * before any capture). */
int p3t_hard_step_vjp(p3t_ctx *ctx, const p3t_particles *p, const p3t_clusters *cl, double dt,
                      double *lx, double *ly, double *lz, double *lvx, double *lvy, double *lvz,
                      double *gm, void *stream);

/* The adjoint of the Kepler drift of every particle of p by dt
 * (the drift's map, mu = G M_*): on entry lx..lvz hold the adjoint of the state
 * after the drift, on return the adjoint of the state before it (Phi^T lam,
 * Phi the state-transition matrix at the state p holds, which is the state
 * BEFORE the drift).  Device arrays, n each, caller order. */
int p3t_kepler_vjp(p3t_ctx *ctx, const p3t_particles *p, double dt, double *lx, double *ly,
                   double *lz, double *lvx, double *lvy, double *lvz, void *stream);

/* Total energy (Eqs. soft and hard; W + (1 - W) = 1 makes it the
 * Newtonian energy): out = device double[4] {E, kinetic, star potential,
 * pair potential}.  The pair sum is direct O(n^2), in FP64 for P3T_FP64 and
 * as FP32 terms on float-float relative coordinates with float-float sums for
 * P3T_MIXED. */
int p3t_energy(p3t_ctx *ctx, const p3t_particles *p, double *out, void *stream);

/* Copies cluster views (from p3t_neighbours, or caller-built) into caller
 * buffers, ordered on `stream`: label, singles, cl_mem int32[n], cl_off
 * int64[n + 1], counts int64[4] (device pointers; entries past the counts are
 * unspecified).  The paper has no counterpart: it exists so that callers can
 * keep the clusters beyond the next p3t_neighbours call. */
int p3t_copy_clusters(p3t_ctx *ctx, const p3t_clusters *cl, int64_t n,
                      int32_t *label, int32_t *singles, int64_t *cl_off,
                      int32_t *cl_mem, int64_t *counts, void *stream);

/* Limits of the bounded device loops and a per-member record of the
 * Hermite block steps (the paper has no counterpart: diagnostics).
 *  - hermite_block_limit: block times one cluster may take in one
 *    p3t_hard_step; a cluster that needs more stops where it is and
 *    P3T_ERR_TIMEOUT is recorded.  0 selects the default, 2^24.
 *  - scan_poll_limit: polls a tile of the library's single-pass scans makes
 *    for its predecessors' sums before it gives up (P3T_ERR_TIMEOUT; the
 *    scan's result is then invalid).  0 selects the default, 2^22.
 *  - hermite_steps: NULL, or a device int32[n] (caller order) into which
 *    every later p3t_hard_step writes, for each member of a cluster of >= 2,
 *    the number of corrector steps the member took; entries of isolated
 *    particles are left as they are.  It must stay valid while it is set and
 *    hold n entries for every later hard step.
 * Host call, no device work; takes effect for work enqueued after it and
 * holds until the next call.  P3T_ERR_INVALID for a NULL argument or a
 * negative limit. */
typedef struct {
  int64_t hermite_block_limit;
  int64_t scan_poll_limit;
  int32_t *hermite_steps;
} p3t_diag;
int p3t_set_diag(p3t_ctx *ctx, const p3t_diag *d);

/* Launch shapes that change speed but not results (the paper has no
 * counterpart: tuning knobs, e.g. for an autotuner).
 *  - hermite_warp_max: clusters of 2..hermite_warp_max members are integrated
 *    by one warp each, larger ones (up to 128) by a block of four warps;
 *    2..32, 0 selects the default 8.
 *  - walk_blocks_per_sm: blocks of the soft-force walk per SM, 1..6 (the
 *    kernel is compiled for 6 resident), 0 selects as many as fit.
 * Host call, no device work; takes effect for work enqueued after it.
 * P3T_ERR_INVALID for a NULL argument or a value out of range. */
typedef struct {
  int32_t hermite_warp_max;
  int32_t walk_blocks_per_sm;
} p3t_tuning;
int p3t_set_tuning(p3t_ctx *ctx, const p3t_tuning *t);

/* Synchronises the context's device, returns the first device-side error
 * recorded since the last call (or 0) and clears it.  *required (may be NULL)
 * receives the buffer size a P3T_ERR_CAPACITY asked for.  Not capturable. */
int p3t_status(p3t_ctx *ctx, int64_t *required);

/* Synchronising read of the last tree: out[4] = {nodes, leaves, deepest level,
 * largest leaf}.  Host memory.  Not capturable. */
int p3t_tree_stats(p3t_ctx *ctx, int64_t out[4]);

/* Number of kernels the library has launched in this process (all contexts);
 * a diagnostic for counting launches per step.  Host only, thread-safe. */
int64_t p3t_launch_count(void);

/* Human-readable text for a status code. */
const char *p3t_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* P3T_H */
