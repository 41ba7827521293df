/*
 * p3t_oracle.h -- plain FP64 CPU oracle for the P3T soft step with individual
 * cut-off radii (Ishigaki et al. 2021, "GPLUM", PASJ 73, 660).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it and shares no code,
 * header, table or constant with it.
 *
 * Conventions: structure-of-arrays FP64, particle indices are the caller's
 * order, int64 CSR offsets, int32 indices.  G and M_* are parameters (the paper
 * uses G = M_* = 1, Sec. 3.1).  Every routine is a straight transcription of a
 * definition or of the paper's procedure; none is blocked, fused or reordered
 * for speed.  Compiled with -ffp-contract=off so that no a*b+c is fused.
 */
#ifndef P3T_ORACLE_H
#define P3T_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double G, m_star;     /* gravitational constant, central-star mass            */
  double dt_soft;       /* soft step Delta t (Eq. HamiltonSol)                   */
  double gamma;         /* r_in / r_out (Sec. 2.1.1)                             */
  double rcut0, rcut1;  /* R~cut,0 and R~cut,1 (Eq. routi2)                      */
  double rs0, rs1, rs2, rs3; /* R~search,0..3 (Eqs. rsearch, rsearch1)           */
  double theta;         /* Barnes-Hut opening angle                              */
  double eta, eta0;     /* Hermite accuracy parameters (Sec. 3.1)                */
  double f_radius;      /* radius enhancement factor f of the collision test     */
                        /* (Sec. 2.4.1; the paper uses 1); 0: no collisions      */
  int32_t leaf_size;    /* maximum particles per leaf / target group             */
  int32_t precision;    /* unused by the oracle (always FP64)                    */
  int32_t vran_bins;    /* radial bins for v_ran; 0 = clamp(N/1000, 1, 1024)     */
  int32_t group_size;   /* target groups: highest nodes holding <= group_size
                           particles (0: every leaf is a group)               */
  int32_t cutoff_mode;  /* 0: Hill + random velocity, individual (Eq. routi2) */
                        /* 1: Hill only, individual (Eq. routi)               */
                        /* 2: shared, max over particles of Eq. routi (rout1) */
} or_params;

/* ---- changeover functions (Sec. 2.1.1, Eq. cutfuncW and the K definition) -- */
double or_changeover_K(double y, double gamma);
double or_changeover_dKdy(double y, double gamma);

/* ---- cut-off and search radii (Eqs. routi2, rsearch) --------------------- */
int or_cutoffs(int64_t n, const double *x, const double *y, const double *z,
               const double *vx, const double *vy, const double *vz,
               const double *m, const or_params *p,
               double *r_out, double *r_search, double *v_ran, int32_t *bin);

/* ---- direct O(N^2) changeover soft force (Eq. softforce) ----------------- */
int or_direct_soft(int64_t n, const double *x, const double *y, const double *z,
                   const double *m, const double *r_out, const or_params *p,
                   double *ax, double *ay, double *az);

/* ---- Morton keys, octree, tree walk (Sec. 2.1.2, Eq. softforce) ---------- */
int or_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                   uint64_t *key, double box_out[4]);
int or_tree_soft(int64_t n, const double *x, const double *y, const double *z,
                 const double *m, const double *r_out, const double *r_search,
                 const or_params *p, int64_t n_targets, const int64_t *targets,
                 double *ax, double *ay, double *az, uint64_t counts[2],
                 int64_t cand_cap, int32_t *cand_i, int32_t *cand_j,
                 int64_t *n_cand, int64_t tree_stats[4]);

/* the Barnes-Hut threshold of a level, ceil((2^(22-level))^2 / theta^2)     */
/* (half cell units, exact), and the node-opening test of reading C4 for a  */
/* group and a node given by their grid boxes (1: open)                     */
int64_t or_bh_threshold(double theta, int level);
int or_mac_open(double theta, int level, const int64_t node_c2[3],
                const int64_t node_qlo[3], const int64_t node_qhi[3], int64_t node_R,
                const int64_t grp_qlo[3], const int64_t grp_qhi[3], int64_t grp_R);

/* the walk's interaction lists: groups, their accepted nodes (kind 0) and  */
/* opened leaves (kind 1) in walk order, node member ranges, sorted order    */
int or_tree_lists(int64_t n, const double *x, const double *y, const double *z,
                  const double *m, const double *r_out, const double *r_search,
                  const or_params *p, const int64_t caps[3], int64_t sizes[3],
                  int64_t *ord, int64_t *node_first, int64_t *node_count,
                  int64_t *group_node, int64_t *group_off, int32_t *rec_kind,
                  int32_t *rec_node);

/* multipole moments of a particle set and their field at a point (Barnes-Hut
 * node term, monopole + traceless quadrupole) */
void or_node_moments(int64_t n, const double *x, const double *y,
                     const double *z, const double *m, double out[10]);
void or_multipole_acc(const double mom[10], double G, double px, double py,
                      double pz, double acc[3]);

/* ---- neighbour filter (Eqs. rsearch, rsearch1, t_min) -------------------- */
int or_neighbour_pair(int64_t i, int64_t j, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy,
                      const double *vz, const double *m, const double *r_out,
                      const double *r_search, const or_params *p);
int64_t or_neighbours_from_candidates(
    int64_t n, const double *x, const double *y, const double *z,
    const double *vx, const double *vy, const double *vz, const double *m,
    const double *r_out, const double *r_search, const or_params *p,
    int64_t n_cand, const int32_t *cand_i, const int32_t *cand_j,
    int64_t *nb_off, int32_t *nb_idx, int64_t nb_cap);
int64_t or_neighbours_brute(int64_t n, const double *x, const double *y,
                            const double *z, const double *vx, const double *vy,
                            const double *vz, const double *m,
                            const double *r_out, const double *r_search,
                            const or_params *p, int64_t *nb_off,
                            int32_t *nb_idx, int64_t nb_cap);

/* ---- neighbour clusters (Sec. 2.3, steps i-iii) --------------------------- */
int64_t or_clusters(int64_t n, const int64_t *nb_off, const int32_t *nb_idx,
                    int32_t *label, int64_t *n_single, int32_t *singles,
                    int64_t *n_clusters, int64_t *cl_off, int32_t *cl_mem);

/* ---- soft kick (procedure steps 3 and 8) ---------------------------------- */
void or_kick(int64_t n, double *vx, double *vy, double *vz, const double *ax,
             const double *ay, const double *az, double h);

/* ---- Hermite-4 hard step of one neighbour cluster ------------------------- */
void or_hard_acc_jerk(int64_t nc, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy,
                      const double *vz, const double *m, const double *r_out,
                      const or_params *p, int64_t k, double acc[3],
                      double jerk[3]);
int or_hermite_cluster(int64_t nc, const int32_t *members, double *x, double *y,
                       double *z, double *vx, double *vy, double *vz,
                       const double *m, const double *r_out, const double *r_phys,
                       const or_params *p, double dt, int64_t *n_steps,
                       int32_t *root_out, double *e_disp, int32_t *member_steps);

/* ---- Kepler drift of isolated particles ----------------------------------- */
int or_kepler_drift(int64_t n, const int32_t *idx, double *x, double *y,
                    double *z, double *vx, double *vy, double *vz, double dt,
                    double mu);

/* ---- Hermite step and Kepler drift together: the hard part of a soft step - */
/* r_phys: physical radii (NULL or f_radius == 0: no collisions); comp_root:   */
/* n entries (or NULL), lowest member of each particle's composite or -1;     */
/* e_hard: energy dissipated by the collisions; member_steps: n entries (or  */
/* NULL), the corrector steps each cluster member took (0 for singles).      */
int or_hard_step(int64_t n, double *x, double *y, double *z, double *vx,
                 double *vy, double *vz, const double *m, const double *r_out,
                 const double *r_phys, const or_params *p, double dt,
                 int64_t n_single, const int32_t *singles, int64_t n_clusters,
                 const int64_t *cl_off, const int32_t *cl_mem,
                 int64_t *n_hermite_steps, int32_t *comp_root, double *e_hard,
                 int32_t *member_steps);

/* ---- composite kick and merge (Sec. 2.4.1, procedure step 9) -------------- */
double or_kick_composites(int64_t n, double *vx, double *vy, double *vz,
                          const double *ax, const double *ay, const double *az,
                          double h, const double *m, const int32_t *comp_root);
int64_t or_merge(int64_t n, double *x, double *y, double *z, double *vx, double *vy,
                 double *vz, double *m, double *r_phys, double *r_out,
                 double *r_search, const int32_t *comp_root, int32_t *new_index);

/* ---- total energy (Eqs. soft + hard with W + (1-W) = 1) ------------------ */
void or_energy(int64_t n, const double *x, const double *y, const double *z,
               const double *vx, const double *vy, const double *vz,
               const double *m, double G, double m_star, double out[4]);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
