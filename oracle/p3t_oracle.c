/*
 * p3t_oracle.c -- plain FP64 CPU oracle for the P3T soft step with individual
 * cut-off radii (Ishigaki et al. 2021).  TEST INFRASTRUCTURE ONLY: loaded by the
 * tests, the smoke check and the benchmark's CPU-baseline leg, never by the
 * product path.  Plain C11 + OpenMP, FP64, built with -ffp-contract=off.
 *
 * Every function states the passage it follows.  Where the paper is silent or
 * garbled, the reading used (numbered C1..C11) is stated beside the code it
 * governs.
 */
#include "p3t_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* ========================================================================= */
/* Changeover functions, Sec. 2.1.1.                                          */
/* The paper prints W(y; gamma) (Eq. cutfuncW) and defines K through          */
/* W(r) = r * int_r^inf K(s)/s^2 ds, so K = W - y dW/dy.  Carrying out the    */
/* derivative of the printed middle branch (reading C1: the garbled term is   */
/* -(10/3) y^7) gives K(y) = S(x), x = (y - gamma)/(1 - gamma), with          */
/* S(x) = 35x^4 - 84x^5 + 70x^6 - 20x^7, K = 0 below gamma and 1 above 1.      */
/* ========================================================================= */
double or_changeover_K(double y, double gamma) {
  if (y <= gamma) return 0.0;
  if (y >= 1.0) return 1.0;
  double x = (y - gamma) / (1.0 - gamma);
  double x2 = x * x;
  double x3 = x2 * x;
  double x4 = x2 * x2;
  return x4 * (35.0 - 84.0 * x + 70.0 * x2 - 20.0 * x3);
}

/* dK/dy = S'(x) / (1 - gamma), S'(x) = 140 x^3 (1 - x)^3 (needed for the jerk
 * of the hard force, Eq. hardforce). */
double or_changeover_dKdy(double y, double gamma) {
  if (y <= gamma || y >= 1.0) return 0.0;
  double x = (y - gamma) / (1.0 - gamma);
  double u = 1.0 - x;
  return 140.0 * x * x * x * u * u * u / (1.0 - gamma);
}

/* ========================================================================= */
/* Cut-off and search radii.                                                  */
/* r_Hill,i = (m_i / 3M_*)^(1/3) a_i (Sec. 2.1.1), a_i the osculating         */
/* semi-major axis; r_out,i = max(R~cut,0 r_Hill,i, R~cut,1 v_ran,i dt)       */
/* (Eq. routi2); r_search,i = R~s,0 r_out,i + R~s,1 v_ran,i dt (Eq. rsearch). */
/* v_ran,i: reading C3 -- random velocity u = v - sqrt(G M_* / r) phi_hat,      */
/* v_ran = sqrt(<|u|^2>) over the particle's radial bin; bins uniform in      */
/* ln R_cyl between the smallest and largest R_cyl.                          */
/* ========================================================================= */
int or_cutoffs(int64_t n, const double *x, const double *y, const double *z,
               const double *vx, const double *vy, const double *vz,
               const double *m, const or_params *p, double *r_out,
               double *r_search, double *v_ran, int32_t *bin) {
  if (n <= 0) return 0;
  const double mu = p->G * p->m_star;
  int64_t nb = p->vran_bins;
  if (nb <= 0) {
    nb = n / 1000;
    if (nb < 1) nb = 1;
    if (nb > 1024) nb = 1024;
  }
  double *R = (double *)malloc(sizeof(double) * n);
  double *u2 = (double *)malloc(sizeof(double) * n);
  double *sum = (double *)calloc(nb, sizeof(double));
  int64_t *cnt = (int64_t *)calloc(nb, sizeof(int64_t));
  int32_t *b = bin ? bin : (int32_t *)malloc(sizeof(int32_t) * n);
  double Rmin = INFINITY, Rmax = -INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    R[i] = sqrt(x[i] * x[i] + y[i] * y[i]);
    if (R[i] < Rmin) Rmin = R[i];
    if (R[i] > Rmax) Rmax = R[i];
    double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    double vk = sqrt(mu / r);
    double px = 0.0, py = 0.0;
    if (R[i] > 0.0) { px = -y[i] / R[i]; py = x[i] / R[i]; }
    double ux = vx[i] - vk * px, uy = vy[i] - vk * py, uz = vz[i];
    u2[i] = ux * ux + uy * uy + uz * uz;
  }
  double lmin = log(Rmin), lmax = log(Rmax);
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = 0;
    if (Rmax > Rmin && R[i] > Rmin) {
      double t = (log(R[i]) - lmin) / (lmax - lmin);
      k = (int64_t)floor(t * (double)nb);
      if (k < 0) k = 0;
      if (k > nb - 1) k = nb - 1;
    }
    b[i] = (int32_t)k;
    sum[k] += u2[i];
    cnt[k] += 1;
  }
  for (int64_t i = 0; i < n; ++i) {
    double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
    double alpha = 2.0 / r - v2 / mu; /* 1/a from the vis-viva relation */
    double a = alpha > 0.0 ? 1.0 / alpha : r;
    double rhill = cbrt(m[i] / (3.0 * p->m_star)) * a;
    double vr = sqrt(sum[b[i]] / (double)cnt[b[i]]);
    if (v_ran) v_ran[i] = vr;
    /* Eq. routi2 (mode 0) or Eq. routi (modes 1, 2); Eq. rsearch */
    double ro = p->cutoff_mode == 0 ? dmax(p->rcut0 * rhill, p->rcut1 * vr * p->dt_soft)
                                    : p->rcut0 * rhill;
    r_out[i] = ro;
    r_search[i] = p->rs0 * ro + p->rs1 * vr * p->dt_soft;
  }
  if (p->cutoff_mode == 2) {
    /* shared cut-off (Eq. rout1): every particle gets the largest r_out, and
     * the largest search radius (Sec. 2.3) */
    double mo = 0.0, ms = 0.0;
    for (int64_t i = 0; i < n; ++i) { mo = dmax(mo, r_out[i]); ms = dmax(ms, r_search[i]); }
    for (int64_t i = 0; i < n; ++i) { r_out[i] = mo; r_search[i] = ms; }
  }
  if (!bin) free(b);
  free(R); free(u2); free(sum); free(cnt);
  return 0;
}

/* ========================================================================= */
/* Direct O(N^2) soft force, Eq. softforce:                                   */
/*   a_i = -sum_{j != i} G m_j K(r_ij; r_out,ij) r_ij / r_ij^3,               */
/*   r_out,ij = max(r_out,i, r_out,j) (Eq. rout2).                            */
/* ========================================================================= */
int or_direct_soft(int64_t n, const double *x, const double *y, const double *z,
                   const double *m, const double *r_out, const or_params *p,
                   double *ax, double *ay, double *az) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double rx = x[i] - x[j], ry = y[i] - y[j], rz = z[i] - z[j];
      double r2 = rx * rx + ry * ry + rz * rz;
      double r = sqrt(r2);
      double ro = dmax(r_out[i], r_out[j]);
      double K = or_changeover_K(r / ro, p->gamma);
      if (K == 0.0) continue;
      double f = p->G * m[j] * K / (r2 * r);
      sx -= f * rx; sy -= f * ry; sz -= f * rz;
    }
    ax[i] = sx; ay[i] = sy; az[i] = sz;
  }
  return 0;
}

/* ========================================================================= */
/* The Barnes-Hut tree (Sec. 2.1.2 uses FDPS's tree; the discrete            */
/* definitions below are reading C4).                                         */
/*  * root cube: bounding box of the positions, made cubic (side L = largest  */
/*    extent), corner at the per-axis minimum;                                */
/*  * each axis quantised to its cell q = floor(d / u), d = v - lo (rounded   */
/*    to FP64), u = L / 2^21 (exact), the quotient taken exactly: the largest */
/*    q with q u <= d, clamped to [0, 2^21); bits interleaved (x highest)     */
/*    into a 63-bit Morton key; particles ordered by (key, caller index);     */
/*  * a node is a key prefix at level l holding > 0 particles; a node is      */
/*    split while it holds more than leaf_size particles and l < 21;          */
/*  * target groups: a node is a group iff it holds <= group_size particles  */
/*    or is a leaf, and it is the root or its parent holds > group_size       */
/*    (group_size = 0: every leaf is a group).  Opening is decided for the    */
/*    group's box on the quantised grid, in exact integer arithmetic:         */
/*    (i) Barnes-Hut: with the node's cell side s and centre c, and the       */
/*        group's cells [qlo, qhi + 1] (all in half units), open iff          */
/*        d^2 < ceil((2 s)^2 / theta^2), d the point-box distance;  this is   */
/*        side^2 > theta^2 d^2 on the grid;                                   */
/*    (ii) cut-off reach: per axis gap g = max(0, qlo_b - qhi_a - 2, ...)     */
/*        (a lower bound of the true gap in units of u), R = ceil(rsmax/u)+1  */
/*        per node; open iff g^2 < max(R_group, R_node)^2.  Every pair closer */
/*        than max(r_search,i, r_search,j) therefore meets in an opened leaf. */
/*    Accepted nodes add monopole + quadrupole; opened leaves add pairs.      */
/* ========================================================================= */
#define OR_BITS 21
#define OR_QMAX ((int64_t)1 << OR_BITS)

static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < OR_BITS; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

static int64_t quantise(double v, double lo, double L) {
  const double u = ldexp(L, -OR_BITS);
  const double d = v - lo;
  int64_t q = (int64_t)floor(d / u);
  /* the rounded quotient can reach the next integer from below: keep q u <= d */
  /* (the fused q u - d is rounded once, so its sign is that of the exact one) */
  if (fma((double)q, u, -d) > 0.0) --q;
  if (q < 0) q = 0;
  if (q > OR_QMAX - 1) q = OR_QMAX - 1;
  return q;
}

static void root_box(int64_t n, const double *x, const double *y,
                     const double *z, double box[4]) {
  double lo[3] = {INFINITY, INFINITY, INFINITY};
  double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i) {
    lo[0] = dmin(lo[0], x[i]); hi[0] = dmax(hi[0], x[i]);
    lo[1] = dmin(lo[1], y[i]); hi[1] = dmax(hi[1], y[i]);
    lo[2] = dmin(lo[2], z[i]); hi[2] = dmax(hi[2], z[i]);
  }
  double L = dmax(hi[0] - lo[0], dmax(hi[1] - lo[1], hi[2] - lo[2]));
  if (!(L > 0.0)) L = 1.0;
  box[0] = lo[0]; box[1] = lo[1]; box[2] = lo[2]; box[3] = L;
}

int or_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                   uint64_t *key, double box_out[4]) {
  double box[4];
  root_box(n, x, y, z, box);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t qx = (uint64_t)quantise(x[i], box[0], box[3]);
    uint64_t qy = (uint64_t)quantise(y[i], box[1], box[3]);
    uint64_t qz = (uint64_t)quantise(z[i], box[2], box[3]);
    key[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
  }
  if (box_out) memcpy(box_out, box, sizeof(box));
  return 0;
}

typedef struct {
  int level;
  int64_t first, count;  /* range in the sorted particle order */
  int64_t child0, nchild; /* children are contiguous in the node array */
  double M, com[3], Q[6]; /* Q = sum m (3 d_a d_b - d^2 delta_ab): xx yy zz xy xz yz */
  double lo[3], hi[3];    /* tight box of the particle positions */
  double rsmax;           /* max r_search over the node's particles */
  int64_t qlo[3], qhi[3]; /* quantised tight box (cells) of the particles */
  int64_t c2[3];          /* cell centre of the node, in half units of u */
  int64_t R;              /* ceil(rsmax / u) + 1, clamped to 2^23 */
} or_node;

typedef struct {
  int64_t n;
  int64_t *ord;      /* sorted position -> caller index */
  uint64_t *key;     /* keys in sorted order */
  double *x, *y, *z, *m, *ro, *rs; /* sorted copies */
  int64_t *qx, *qy, *qz;
  or_node *node;
  int64_t nnode, cap;
  int64_t *parent;   /* parent node, -1 for the root */
  double box[4];
} or_tree;

typedef struct { uint64_t key; int64_t idx; } kv_t;
static int cmp_kv(const void *a, const void *b) {
  const kv_t *u = (const kv_t *)a, *v = (const kv_t *)b;
  if (u->key != v->key) return u->key < v->key ? -1 : 1;
  return (u->idx > v->idx) - (u->idx < v->idx);
}

/* Moments of a particle set straight from the definitions: M = sum m,        */
/* com = sum m x / M, Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab), d = x - com. */
void or_node_moments(int64_t n, const double *x, const double *y,
                     const double *z, const double *m, double out[10]) {
  double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    M += m[i]; sx += m[i] * x[i]; sy += m[i] * y[i]; sz += m[i] * z[i];
  }
  double cx = sx / M, cy = sy / M, cz = sz / M;
  double Q[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    double dx = x[i] - cx, dy = y[i] - cy, dz = z[i] - cz;
    double d2 = dx * dx + dy * dy + dz * dz;
    Q[0] += m[i] * (3.0 * dx * dx - d2);
    Q[1] += m[i] * (3.0 * dy * dy - d2);
    Q[2] += m[i] * (3.0 * dz * dz - d2);
    Q[3] += m[i] * (3.0 * dx * dy);
    Q[4] += m[i] * (3.0 * dx * dz);
    Q[5] += m[i] * (3.0 * dy * dz);
  }
  out[0] = M; out[1] = cx; out[2] = cy; out[3] = cz;
  for (int k = 0; k < 6; ++k) out[4 + k] = Q[k];
}

/* Field of a monopole + quadrupole at p: the potential of the set is          */
/* phi = -G [M/r + (r.Q.r)/(2 r^5)], r = p - com, so                            */
/* a = -grad phi = G [-M r/r^3 + Q.r/r^5 - (5/2)(r.Q.r) r/r^7].                */
void or_multipole_acc(const double mom[10], double G, double px, double py,
                      double pz, double acc[3]) {
  double dx = px - mom[1], dy = py - mom[2], dz = pz - mom[3];
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
  const double *Q = mom + 4;
  double qx = Q[0] * dx + Q[3] * dy + Q[4] * dz;
  double qy = Q[3] * dx + Q[1] * dy + Q[5] * dz;
  double qz = Q[4] * dx + Q[5] * dy + Q[2] * dz;
  double rqr = dx * qx + dy * qy + dz * qz;
  double M = mom[0];
  acc[0] = G * (-M * dx / r3 + qx / r5 - 2.5 * rqr * dx / r7);
  acc[1] = G * (-M * dy / r3 + qy / r5 - 2.5 * rqr * dy / r7);
  acc[2] = G * (-M * dz / r3 + qz / r5 - 2.5 * rqr * dz / r7);
}

static int64_t push_node(or_tree *T) {
  if (T->nnode == T->cap) {
    T->cap = T->cap ? 2 * T->cap : 1024;
    T->node = (or_node *)realloc(T->node, sizeof(or_node) * T->cap);
  }
  memset(&T->node[T->nnode], 0, sizeof(or_node));
  return T->nnode++;
}

static void fill_node(or_tree *T, or_node *nd) {
  int64_t f = nd->first, c = nd->count;
  double mom[10];
  or_node_moments(c, T->x + f, T->y + f, T->z + f, T->m + f, mom);
  nd->M = mom[0];
  for (int k = 0; k < 3; ++k) nd->com[k] = mom[1 + k];
  for (int k = 0; k < 6; ++k) nd->Q[k] = mom[4 + k];
  for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
  nd->rsmax = 0.0;
  for (int64_t i = f; i < f + c; ++i) {
    nd->lo[0] = dmin(nd->lo[0], T->x[i]); nd->hi[0] = dmax(nd->hi[0], T->x[i]);
    nd->lo[1] = dmin(nd->lo[1], T->y[i]); nd->hi[1] = dmax(nd->hi[1], T->y[i]);
    nd->lo[2] = dmin(nd->lo[2], T->z[i]); nd->hi[2] = dmax(nd->hi[2], T->z[i]);
    nd->rsmax = dmax(nd->rsmax, T->rs[i]);
  }
  /* quantised box, cell centre and search reach on the grid */
  for (int a = 0; a < 3; ++a) { nd->qlo[a] = OR_QMAX; nd->qhi[a] = -1; }
  for (int64_t i = f; i < f + c; ++i) {
    const int64_t q[3] = {T->qx[i], T->qy[i], T->qz[i]};
    for (int a = 0; a < 3; ++a) {
      if (q[a] < nd->qlo[a]) nd->qlo[a] = q[a];
      if (q[a] > nd->qhi[a]) nd->qhi[a] = q[a];
    }
  }
  int sh = OR_BITS - nd->level;
  nd->c2[0] = (2 * (T->qx[f] >> sh) + 1) << sh;
  nd->c2[1] = (2 * (T->qy[f] >> sh) + 1) << sh;
  nd->c2[2] = (2 * (T->qz[f] >> sh) + 1) << sh;
  double u = ldexp(T->box[3], -OR_BITS);
  double rq = ceil(nd->rsmax / u) + 1.0;
  nd->R = rq < 8388608.0 ? (int64_t)rq : 8388608;
}

static void tree_build(or_tree *T, int64_t n, const double *x, const double *y,
                       const double *z, const double *m, const double *ro,
                       const double *rs, int leaf) {
  memset(T, 0, sizeof(*T));
  T->n = n;
  uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * n);
  or_morton_keys(n, x, y, z, key, T->box);
  kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * n);
  for (int64_t i = 0; i < n; ++i) { kv[i].key = key[i]; kv[i].idx = i; }
  qsort(kv, n, sizeof(kv_t), cmp_kv);
  T->ord = (int64_t *)malloc(sizeof(int64_t) * n);
  T->key = (uint64_t *)malloc(sizeof(uint64_t) * n);
  T->x = (double *)malloc(sizeof(double) * n);
  T->y = (double *)malloc(sizeof(double) * n);
  T->z = (double *)malloc(sizeof(double) * n);
  T->m = (double *)malloc(sizeof(double) * n);
  T->ro = (double *)malloc(sizeof(double) * n);
  T->rs = (double *)malloc(sizeof(double) * n);
  T->qx = (int64_t *)malloc(sizeof(int64_t) * n);
  T->qy = (int64_t *)malloc(sizeof(int64_t) * n);
  T->qz = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t s = 0; s < n; ++s) {
    int64_t i = kv[s].idx;
    T->ord[s] = i; T->key[s] = kv[s].key;
    T->x[s] = x[i]; T->y[s] = y[i]; T->z[s] = z[i]; T->m[s] = m[i];
    T->ro[s] = ro[i]; T->rs[s] = rs[i];
    T->qx[s] = quantise(x[i], T->box[0], T->box[3]);
    T->qy[s] = quantise(y[i], T->box[1], T->box[3]);
    T->qz[s] = quantise(z[i], T->box[2], T->box[3]);
  }
  free(kv); free(key);
  /* breadth-first: children of a node are appended contiguously */
  int64_t r = push_node(T);
  T->node[r].level = 0; T->node[r].first = 0; T->node[r].count = n;
  for (int64_t k = 0; k < T->nnode; ++k) {
    or_node nd = T->node[k];
    if (nd.count > leaf && nd.level < OR_BITS) {
      int sh = 3 * (OR_BITS - (nd.level + 1));
      int64_t c0 = T->nnode, nc = 0;
      int64_t s = nd.first, e = nd.first + nd.count;
      while (s < e) {
        uint64_t d = (T->key[s] >> sh) & 7ull;
        int64_t t = s;
        while (t < e && ((T->key[t] >> sh) & 7ull) == d) ++t;
        int64_t c = push_node(T);
        T->node[c].level = nd.level + 1; T->node[c].first = s;
        T->node[c].count = t - s;
        ++nc;
        s = t;
      }
      T->node[k].child0 = c0; T->node[k].nchild = nc;
    }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < T->nnode; ++k) fill_node(T, &T->node[k]);
  T->parent = (int64_t *)malloc(sizeof(int64_t) * T->nnode);
  T->parent[0] = -1;
  for (int64_t k = 0; k < T->nnode; ++k)
    for (int64_t c = T->node[k].child0; c < T->node[k].child0 + T->node[k].nchild; ++c)
      T->parent[c] = k;
}

static void tree_free(or_tree *T) {
  free(T->ord); free(T->key); free(T->x); free(T->y); free(T->z); free(T->m);
  free(T->ro); free(T->rs); free(T->qx); free(T->qy); free(T->qz);
  free(T->node); free(T->parent);
}

/* Barnes-Hut thresholds per level (reading C4): open iff d^2 < T[l], T[l]   */
/* the smallest integer >= side^2 / theta^2, side = 2^(22-l) half units, so  */
/* that d^2 < T[l] is exactly side^2 > theta^2 d^2 for the integer d^2.       */
/* Exact integer arithmetic: theta = M 2^E with M an odd integer (frexp), so  */
/* side^2 / theta^2 = 2^K / M^2 with K = 2(22 - l) - 2E, and T = ceil(2^K /   */
/* M^2) by long division (M^2 < 2^106, held in 128 bits).  T is capped at     */
/* 2^62, above every d^2 on the grid; theta = 0 opens every node.            */
#define OR_TCAP ((int64_t)1 << 62)
static int64_t bh_threshold(double theta, int level) {
  if (!(theta > 0.0)) return OR_TCAP;
  int e;
  double fr = frexp(theta, &e);              /* theta = fr 2^e, 1/2 <= fr < 1 */
  uint64_t M = (uint64_t)ldexp(fr, 53);      /* theta = M 2^(e - 53) exactly   */
  int E = e - 53;
  while ((M & 1u) == 0) { M >>= 1; ++E; }
  const unsigned __int128 D = (unsigned __int128)M * M;
  const int K = 2 * (OR_BITS + 1 - level) - 2 * E;
  if (K < 0) return 1;                       /* 0 < side^2 / theta^2 < 1 */
  unsigned __int128 r = 0;
  int64_t q = 0;
  for (int b = K; b >= 0; --b) {             /* the bits of 2^K, highest first */
    r = (r << 1) | (unsigned __int128)(b == K);
    int bit = 0;
    if (r >= D) { r -= D; bit = 1; }
    q = 2 * q + bit;
    if (q >= OR_TCAP) return OR_TCAP;
  }
  if (r != 0) ++q;
  return q < OR_TCAP ? q : OR_TCAP;
}

static void bh_thresholds(double theta, int64_t T[OR_BITS + 1]) {
  for (int l = 0; l <= OR_BITS; ++l) T[l] = bh_threshold(theta, l);
}

/* The opening test of a node for a target group, on the grid (reading C4), */
/* exported for the tests: cells [gq_lo, gq_hi] of the group, the node's     */
/* level, cell centre c2 (half units), cells [nq_lo, nq_hi] and the reaches  */
/* R of both.  Returns 1 when the node is opened.                             */
/* Opening decision for node nd seen from target group g (reading C4). */
static int mac_open(const or_node *g, const or_node *nd, const int64_t *bh) {
  int64_t d2 = 0, g2 = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t lo = 2 * g->qlo[a], hi = 2 * g->qhi[a] + 2, d = 0;
    if (nd->c2[a] < lo) d = lo - nd->c2[a];
    else if (nd->c2[a] > hi) d = nd->c2[a] - hi;
    d2 += d * d;
    int64_t gap = 0;
    if (nd->qlo[a] - g->qhi[a] - 2 > gap) gap = nd->qlo[a] - g->qhi[a] - 2;
    if (g->qlo[a] - nd->qhi[a] - 2 > gap) gap = g->qlo[a] - nd->qhi[a] - 2;
    g2 += gap * gap;
  }
  if (d2 < bh[nd->level]) return 1;
  int64_t R = g->R > nd->R ? g->R : nd->R;
  return g2 < R * R;
}

int or_mac_open(double theta, int level, const int64_t node_c2[3],
                const int64_t node_qlo[3], const int64_t node_qhi[3], int64_t node_R,
                const int64_t grp_qlo[3], const int64_t grp_qhi[3], int64_t grp_R) {
  or_node g, nd;
  memset(&g, 0, sizeof(g));
  memset(&nd, 0, sizeof(nd));
  for (int a = 0; a < 3; ++a) {
    g.qlo[a] = grp_qlo[a]; g.qhi[a] = grp_qhi[a];
    nd.qlo[a] = node_qlo[a]; nd.qhi[a] = node_qhi[a]; nd.c2[a] = node_c2[a];
  }
  g.R = grp_R; nd.R = node_R; nd.level = level;
  int64_t bh[OR_BITS + 1];
  bh_thresholds(theta, bh);
  return mac_open(&g, &nd, bh);
}

int64_t or_bh_threshold(double theta, int level) { return bh_threshold(theta, level); }

typedef struct {
  int32_t *ci, *cj;
  int64_t n, cap;
} cand_buf;

static void cand_push(cand_buf *b, int32_t i, int32_t j) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 256;
    b->ci = (int32_t *)realloc(b->ci, sizeof(int32_t) * b->cap);
    b->cj = (int32_t *)realloc(b->cj, sizeof(int32_t) * b->cap);
  }
  b->ci[b->n] = i; b->cj[b->n] = j; b->n++;
}

typedef struct {
  const or_tree *T;
  const or_params *p;
  const or_node *g;
  const unsigned char *is_target;
  double (*acc)[3]; /* accumulators of the group's targets (indexed s - first) */
  uint64_t npp, npn;
  cand_buf *cb;
  const int64_t *bh;
  cand_buf *rec;    /* or NULL: the group's list as (kind, node): 0 accepted node, 1 opened leaf */
} walk_ctx;

static void walk(walk_ctx *w, int64_t k) {
  const or_tree *T = w->T;
  const or_node *nd = &T->node[k];
  const or_node *g = w->g;
  if (!mac_open(g, nd, w->bh)) {
    if (w->rec) cand_push(w->rec, 0, (int32_t)k);
    double mom[10] = {nd->M, nd->com[0], nd->com[1], nd->com[2], nd->Q[0],
                      nd->Q[1], nd->Q[2], nd->Q[3], nd->Q[4], nd->Q[5]};
    for (int64_t s = g->first; s < g->first + g->count; ++s) {
      if (!w->is_target[s]) continue;
      double a[3];
      or_multipole_acc(mom, w->p->G, T->x[s], T->y[s], T->z[s], a);
      double *acc = w->acc[s - g->first];
      acc[0] += a[0]; acc[1] += a[1]; acc[2] += a[2];
      w->npn += 1;
    }
    return;
  }
  if (nd->nchild == 0) {
    if (w->rec) cand_push(w->rec, 1, (int32_t)k);
    for (int64_t s = g->first; s < g->first + g->count; ++s) {
      if (!w->is_target[s]) continue;
      double *acc = w->acc[s - g->first];
      for (int64_t t = nd->first; t < nd->first + nd->count; ++t) {
        if (t == s) continue;
        w->npp += 1;
        double rx = T->x[s] - T->x[t], ry = T->y[s] - T->y[t], rz = T->z[s] - T->z[t];
        double r2 = rx * rx + ry * ry + rz * rz;
        double rs = dmax(T->rs[s], T->rs[t]);
        if (r2 < rs * rs) cand_push(w->cb, (int32_t)T->ord[s], (int32_t)T->ord[t]);
        double r = sqrt(r2);
        double ro = dmax(T->ro[s], T->ro[t]);
        double K = or_changeover_K(r / ro, w->p->gamma);
        if (K == 0.0) continue;
        double f = w->p->G * T->m[t] * K / (r2 * r);
        acc[0] -= f * rx; acc[1] -= f * ry; acc[2] -= f * rz;
      }
    }
    return;
  }
  for (int64_t c = nd->child0; c < nd->child0 + nd->nchild; ++c) walk(w, c);
}

int or_tree_soft(int64_t n, const double *x, const double *y, const double *z,
                 const double *m, const double *r_out, const double *r_search,
                 const or_params *p, int64_t n_targets, const int64_t *targets,
                 double *ax, double *ay, double *az, uint64_t counts[2],
                 int64_t cand_cap, int32_t *cand_i, int32_t *cand_j,
                 int64_t *n_cand, int64_t tree_stats[4]) {
  if (n <= 0) { if (counts) counts[0] = counts[1] = 0; if (n_cand) *n_cand = 0; return 0; }
  or_tree T;
  tree_build(&T, n, x, y, z, m, r_out, r_search, p->leaf_size);
  unsigned char *is_target = (unsigned char *)calloc(n, 1);
  int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t s = 0; s < n; ++s) inv[T.ord[s]] = s;
  if (targets) {
    for (int64_t k = 0; k < n_targets; ++k) is_target[inv[targets[k]]] = 1;
  } else {
    memset(is_target, 1, n);
  }
  /* target groups (see above), in node order */
  int64_t nleaf = 0, maxdepth = 0, ngroup = 0;
  const int64_t gs = p->group_size;
  int64_t *leaves = (int64_t *)malloc(sizeof(int64_t) * T.nnode);
  for (int64_t k = 0; k < T.nnode; ++k) {
    if (T.node[k].nchild == 0) ++nleaf;
    if (T.node[k].level > maxdepth) maxdepth = T.node[k].level;
    int small = T.node[k].count <= gs || T.node[k].nchild == 0;
    int top = k == 0 || T.node[T.parent[k]].count > gs;
    if (small && top) leaves[ngroup++] = k;
  }
  int nth = or_num_threads();
  cand_buf *cbs = (cand_buf *)calloc(nth, sizeof(cand_buf));
  uint64_t npp = 0, npn = 0;
  int64_t bh[OR_BITS + 1];
  bh_thresholds(p->theta, bh);
#pragma omp parallel reduction(+ : npp, npn)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double (*acc)[3] = (double (*)[3])malloc(sizeof(double) * 3 * (p->leaf_size > 0 ? p->leaf_size : 1) + 3 * sizeof(double) * 64);
#pragma omp for schedule(dynamic, 16)
    for (int64_t gi = 0; gi < ngroup; ++gi) {
      const or_node *g = &T.node[leaves[gi]];
      int any = 0;
      for (int64_t s = g->first; s < g->first + g->count; ++s) any |= is_target[s];
      if (!any) continue;
      /* a group may exceed the preallocated size; grow the accumulator then */
      double (*a)[3] = acc;
      double (*big)[3] = NULL;
      if (g->count > (p->leaf_size > 0 ? p->leaf_size : 1) + 64) {
        big = (double (*)[3])malloc(sizeof(double) * 3 * g->count);
        a = big;
      }
      memset(a, 0, sizeof(double) * 3 * g->count);
      walk_ctx w = {&T, p, g, is_target, a, 0, 0, &cbs[tid], bh, NULL};
      walk(&w, 0);
      for (int64_t s = g->first; s < g->first + g->count; ++s) {
        if (!is_target[s]) continue;
        int64_t i = T.ord[s];
        ax[i] = a[s - g->first][0]; ay[i] = a[s - g->first][1]; az[i] = a[s - g->first][2];
      }
      npp += w.npp; npn += w.npn;
      free(big);
    }
    free(acc);
  }
  int64_t nc = 0;
  for (int t = 0; t < nth; ++t) {
    for (int64_t k = 0; k < cbs[t].n; ++k) {
      if (nc < cand_cap && cand_i && cand_j) { cand_i[nc] = cbs[t].ci[k]; cand_j[nc] = cbs[t].cj[k]; }
      ++nc;
    }
    free(cbs[t].ci); free(cbs[t].cj);
  }
  free(cbs);
  if (n_cand) *n_cand = nc;
  if (counts) { counts[0] = npp; counts[1] = npn; }
  if (tree_stats) {
    tree_stats[0] = T.nnode; tree_stats[1] = nleaf; tree_stats[2] = maxdepth;
    tree_stats[3] = 0;
    for (int64_t k = 0; k < T.nnode; ++k)
      if (T.node[k].nchild == 0 && T.node[k].count > tree_stats[3])
        tree_stats[3] = T.node[k].count;
  }
  free(leaves); free(is_target); free(inv);
  tree_free(&T);
  return 0;
}

/* The interaction lists of the tree walk (the same tree, groups and opening */
/* decisions as or_tree_soft), for the adjoint's oracle: the sorted order   */
/* ord (sorted position -> caller index), every node's member range         */
/* [first, first + count) in sorted order, the target groups (their node)   */
/* and per group its list, in walk order, of accepted nodes (kind 0, whose  */
/* monopole + quadrupole act on the group's particles) and opened leaves    */
/* (kind 1, whose particles act as pairs on every other particle of the     */
/* group).  sizes = {nodes, groups, list entries}; arrays beyond their caps  */
/* (caps, same order) are left unfilled and the caller asks again.          */
int or_tree_lists(int64_t n, const double *x, const double *y, const double *z,
                  const double *m, const double *r_out, const double *r_search,
                  const or_params *p, const int64_t caps[3], int64_t sizes[3],
                  int64_t *ord, int64_t *node_first, int64_t *node_count,
                  int64_t *group_node, int64_t *group_off, int32_t *rec_kind,
                  int32_t *rec_node) {
  sizes[0] = sizes[1] = sizes[2] = 0;
  if (n <= 0) return 0;
  or_tree T;
  tree_build(&T, n, x, y, z, m, r_out, r_search, p->leaf_size);
  unsigned char *none = (unsigned char *)calloc(n, 1);
  int64_t bh[OR_BITS + 1];
  bh_thresholds(p->theta, bh);
  const int64_t gs = p->group_size;
  cand_buf rec = {0, 0, 0, 0};
  int64_t ngroup = 0;
  sizes[0] = T.nnode;
  for (int64_t k = 0; k < T.nnode; ++k) {
    if (k < caps[0]) { node_first[k] = T.node[k].first; node_count[k] = T.node[k].count; }
    int small = T.node[k].count <= gs || T.node[k].nchild == 0;
    int top = k == 0 || T.node[T.parent[k]].count > gs;
    if (!(small && top)) continue;
    if (ngroup < caps[1]) { group_node[ngroup] = k; group_off[ngroup] = rec.n; }
    walk_ctx w = {&T, p, &T.node[k], none, NULL, 0, 0, NULL, bh, &rec};
    walk(&w, 0);
    ++ngroup;
  }
  if (ngroup < caps[1] + 1 && group_off) group_off[ngroup] = rec.n;
  for (int64_t q = 0; q < rec.n && q < caps[2]; ++q) { rec_kind[q] = rec.ci[q]; rec_node[q] = rec.cj[q]; }
  for (int64_t s2 = 0; s2 < n && ord; ++s2) ord[s2] = T.ord[s2];
  sizes[1] = ngroup;
  sizes[2] = rec.n;
  free(rec.ci); free(rec.cj); free(none);
  tree_free(&T);
  return 0;
}

/* ========================================================================= */
/* Neighbour predicate, Sec. 2.3.                                            */
/* Candidates: r_ij < r_search,ij = max(r_search,i, r_search,j) (Eq. rsearch  */
/* and the individual-cut-off rule after it).  A candidate is dropped when    */
/* its closest approach under linear motion over [0, dt] exceeds             */
/* R~s,2 r_out,ij (Eq. rsearch1 with t_min; reading C5: "takes a maximum" is  */
/* read as the minimum the t_min formula computes), unless                    */
/* v_ij < R~s,3 a_ij dt/2 with a_ij = G (m_i + m_j) / r_ij^2.                 */
/* All comparisons on squared FP64 quantities.                               */
/* ========================================================================= */
int or_neighbour_pair(int64_t i, int64_t j, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy,
                      const double *vz, const double *m, const double *r_out,
                      const double *r_search, const or_params *p) {
  double rx = x[i] - x[j], ry = y[i] - y[j], rz = z[i] - z[j];
  double r2 = rx * rx + ry * ry + rz * rz;
  double rs = dmax(r_search[i], r_search[j]);
  if (!(r2 < rs * rs)) return 0;
  double ux = vx[i] - vx[j], uy = vy[i] - vy[j], uz = vz[i] - vz[j];
  double v2 = ux * ux + uy * uy + uz * uz;
  double rv = rx * ux + ry * uy + rz * uz;
  double t = 0.0;
  if (v2 > 0.0) {
    t = -rv / v2;
    if (t < 0.0) t = 0.0;
    if (t >= p->dt_soft) t = p->dt_soft;
  }
  double dx = rx + ux * t, dy = ry + uy * t, dz = rz + uz * t;
  double d2 = dx * dx + dy * dy + dz * dz;
  double lim = p->rs2 * dmax(r_out[i], r_out[j]);
  if (d2 <= lim * lim) return 1;
  double a = p->G * (m[i] + m[j]) / r2;
  double w = p->rs3 * a * p->dt_soft * 0.5;
  return v2 < w * w;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
  return (u > v) - (u < v);
}

/* Assemble CSR rows from accepted (i, j) pairs; rows sorted by j, duplicates */
/* removed.  Returns the number of entries (may exceed nb_cap: then only the  */
/* offsets are valid and the caller retries with a larger capacity).          */
static int64_t build_csr(int64_t n, int64_t npair, const int32_t *pi,
                         const int32_t *pj, int64_t *nb_off, int32_t *nb_idx,
                         int64_t nb_cap) {
  int64_t *cnt = (int64_t *)calloc(n + 1, sizeof(int64_t));
  for (int64_t k = 0; k < npair; ++k) cnt[pi[k]]++;
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (npair > 0 ? npair : 1));
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  pos[0] = 0;
  for (int64_t i = 0; i < n; ++i) pos[i + 1] = pos[i] + cnt[i];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  memcpy(fill, pos, sizeof(int64_t) * (n + 1));
  for (int64_t k = 0; k < npair; ++k) tmp[fill[pi[k]]++] = pj[k];
  int64_t tot = 0;
  nb_off[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t *row = tmp + pos[i];
    int64_t len = pos[i + 1] - pos[i];
    qsort(row, len, sizeof(int32_t), cmp_i32);
    for (int64_t k = 0; k < len; ++k) {
      if (k > 0 && row[k] == row[k - 1]) continue;
      if (tot < nb_cap && nb_idx) nb_idx[tot] = row[k];
      ++tot;
    }
    nb_off[i + 1] = tot;
  }
  free(cnt); free(tmp); free(pos); free(fill);
  return tot;
}

int64_t or_neighbours_from_candidates(
    int64_t n, const double *x, const double *y, const double *z,
    const double *vx, const double *vy, const double *vz, const double *m,
    const double *r_out, const double *r_search, const or_params *p,
    int64_t n_cand, const int32_t *cand_i, const int32_t *cand_j,
    int64_t *nb_off, int32_t *nb_idx, int64_t nb_cap) {
  int32_t *ki = (int32_t *)malloc(sizeof(int32_t) * (n_cand > 0 ? n_cand : 1));
  int32_t *kj = (int32_t *)malloc(sizeof(int32_t) * (n_cand > 0 ? n_cand : 1));
  int64_t nk = 0;
  for (int64_t k = 0; k < n_cand; ++k) {
    if (or_neighbour_pair(cand_i[k], cand_j[k], x, y, z, vx, vy, vz, m, r_out,
                          r_search, p)) {
      ki[nk] = cand_i[k]; kj[nk] = cand_j[k]; ++nk;
    }
  }
  int64_t tot = build_csr(n, nk, ki, kj, nb_off, nb_idx, nb_cap);
  free(ki); free(kj);
  return tot;
}

int64_t or_neighbours_brute(int64_t n, const double *x, const double *y,
                            const double *z, const double *vx, const double *vy,
                            const double *vz, const double *m,
                            const double *r_out, const double *r_search,
                            const or_params *p, int64_t *nb_off,
                            int32_t *nb_idx, int64_t nb_cap) {
  cand_buf b = {0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      if (j != i && or_neighbour_pair(i, j, x, y, z, vx, vy, vz, m, r_out, r_search, p))
        cand_push(&b, (int32_t)i, (int32_t)j);
  int64_t tot = build_csr(n, b.n, b.ci, b.cj, nb_off, nb_idx, nb_cap);
  free(b.ci); free(b.cj);
  return tot;
}

/* ========================================================================= */
/* Neighbour clusters, Sec. 2.3 steps i-iii: every particle starts           */
/* with its own index as cluster index; each particle takes the minimum of    */
/* its own and its neighbours' indices; repeat until nothing changes.  Then   */
/* compaction: isolated particles ascending; clusters of >= 2 members ordered */
/* by label, members ascending.  Returns the size of the largest cluster.     */
/* ========================================================================= */
int64_t or_clusters(int64_t n, const int64_t *nb_off, const int32_t *nb_idx,
                    int32_t *label, int64_t *n_single, int32_t *singles,
                    int64_t *n_clusters, int64_t *cl_off, int32_t *cl_mem) {
  for (int64_t i = 0; i < n; ++i) label[i] = (int32_t)i;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int64_t i = 0; i < n; ++i) {
      int32_t l = label[i];
      for (int64_t k = nb_off[i]; k < nb_off[i + 1]; ++k)
        if (label[nb_idx[k]] < l) l = label[nb_idx[k]];
      if (l < label[i]) { label[i] = l; changed = 1; }
    }
  }
  int64_t *size = (int64_t *)calloc(n > 0 ? n : 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) size[label[i]]++;
  int64_t ns = 0, nc = 0, maxsz = n > 0 ? 1 : 0;
  int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    if (size[label[i]] == 1) { if (singles) singles[ns] = (int32_t)i; ++ns; }
    if (label[i] == i && size[i] >= 2) {
      cid[i] = nc++;
      if (size[i] > maxsz) maxsz = size[i];
    }
  }
  if (cl_off) {
    cl_off[0] = 0;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
      if (label[i] == i && size[i] >= 2) { cl_off[c + 1] = cl_off[c] + size[i]; ++c; }
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    for (int64_t k = 0; k < nc; ++k) fill[k] = cl_off[k];
    for (int64_t i = 0; i < n; ++i)
      if (size[label[i]] >= 2) cl_mem[fill[cid[label[i]]]++] = (int32_t)i;
    free(fill);
  }
  if (n_single) *n_single = ns;
  if (n_clusters) *n_clusters = nc;
  free(size); free(cid);
  return maxsz;
}

/* ========================================================================= */
/* Soft velocity kick v += a_soft * h, h = dt/2 (procedure steps 3           */
/* and 8, Eq. HamiltonSol).                                                   */
/* ========================================================================= */
void or_kick(int64_t n, double *vx, double *vy, double *vz, const double *ax,
             const double *ay, const double *az, double h) {
  for (int64_t i = 0; i < n; ++i) {
    vx[i] += ax[i] * h; vy[i] += ay[i] * h; vz[i] += az[i] * h;
  }
}

/* ========================================================================= */
/* Hard force and jerk on member k of a cluster (Eq. hardforce):             */
/*   a_k = -G M_* x_k / |x_k|^3 - sum_{j != k} G m_j (1 - K(y)) r / r^3,      */
/* r = x_k - x_j, y = r / r_out,kj (reading C8: all other cluster members).   */
/* The jerk is the time derivative along the relative velocity u:            */
/*   d/dt [(1 - K) r / r^3] = (1 - K) [u / r^3 - 3 (r.u) r / r^5]             */
/*                            - K'(y) (r.u) / (r r_out,kj) r / r^3.           */
/* Written as printed, term by term; member sets (composites, Sec. 2.4.1):   */
/* with set given, the other members of k's own composite (set[j] ==          */
/* set[k]) are left out, and with RP given *partner receives the lowest-     */
/* index member j outside k's composite that touches k, r_kj < f (R_p,k +    */
/* R_p,j), at the positions the force is evaluated at (or -1).                */
/* ========================================================================= */
static void hard_acc_jerk_sets(int64_t nc, const double *x, const double *y,
                               const double *z, const double *vx, const double *vy,
                               const double *vz, const double *m, const double *r_out,
                               const double *RP, const int64_t *set, const or_params *p,
                               int64_t k, double acc[3], double jerk[3], int64_t *partner) {
  double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
  if (partner) *partner = -1;
  {
    /* the central star: -G M_* x / r^3 and its derivative */
    double r2 = x[k] * x[k] + y[k] * y[k] + z[k] * z[k];
    double r = sqrt(r2);
    double r3 = r2 * r, r5 = r3 * r2;
    double rv = x[k] * vx[k] + y[k] * vy[k] + z[k] * vz[k];
    double GM = p->G * p->m_star;
    ax -= GM * x[k] / r3; ay -= GM * y[k] / r3; az -= GM * z[k] / r3;
    jx -= GM * (vx[k] / r3 - 3.0 * rv * x[k] / r5);
    jy -= GM * (vy[k] / r3 - 3.0 * rv * y[k] / r5);
    jz -= GM * (vz[k] / r3 - 3.0 * rv * z[k] / r5);
  }
  for (int64_t j = 0; j < nc; ++j) {
    if (j == k || (set && set[j] == set[k])) continue;
    double rx = x[k] - x[j], ry = y[k] - y[j], rz = z[k] - z[j];
    double ux = vx[k] - vx[j], uy = vy[k] - vy[j], uz = vz[k] - vz[j];
    double r2 = rx * rx + ry * ry + rz * rz;
    if (RP && partner && *partner < 0) {
      double sr = p->f_radius * (RP[k] + RP[j]);
      if (r2 < sr * sr) *partner = j;
    }
    if (r2 == 0.0) continue;
    double r = sqrt(r2);
    double ro = dmax(r_out[k], r_out[j]);
    double yv = r / ro;
    double w = 1.0 - or_changeover_K(yv, p->gamma);
    if (w == 0.0) continue;
    double dK = or_changeover_dKdy(yv, p->gamma);
    double r3 = r2 * r, r5 = r3 * r2;
    double rv = rx * ux + ry * uy + rz * uz;
    double Gm = p->G * m[j];
    ax -= Gm * w * rx / r3; ay -= Gm * w * ry / r3; az -= Gm * w * rz / r3;
    double dw = dK * rv / (r * ro); /* -d(1 - K)/dt */
    jx -= Gm * (w * (ux / r3 - 3.0 * rv * rx / r5) - dw * rx / r3);
    jy -= Gm * (w * (uy / r3 - 3.0 * rv * ry / r5) - dw * ry / r3);
    jz -= Gm * (w * (uz / r3 - 3.0 * rv * rz / r5) - dw * rz / r3);
  }
  acc[0] = ax; acc[1] = ay; acc[2] = az;
  jerk[0] = jx; jerk[1] = jy; jerk[2] = jz;
}

void or_hard_acc_jerk(int64_t nc, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy,
                      const double *vz, const double *m, const double *r_out,
                      const or_params *p, int64_t k, double acc[3],
                      double jerk[3]) {
  hard_acc_jerk_sets(nc, x, y, z, vx, vy, vz, m, r_out, NULL, NULL, p, k, acc, jerk, NULL);
}

/* Block time-step quantisation (reading C7): the largest dt_soft / 2^k not   */
/* above the desired step, k <= 40, at most twice the previous step, and      */
/* commensurate with the particle's current time (integer units of           */
/* dt_soft / 2^40).  Sets *underflow when even dt_soft / 2^40 is too long.     */
#define OR_KMAX 40
/* a cluster whose steps collapse (two bodies passing ever closer: the paper
 * merges such pairs, Sec. 2.4) is given up after this many block steps */
#define OR_BLOCK_LIMIT ((int64_t)1 << 24)
static int quantise_level(double dt_des, double dt_soft, int prev_level,
                          int64_t t_int, int *underflow) {
  int lvl = 0;
  while (lvl < OR_KMAX && ldexp(dt_soft, -lvl) > dt_des) ++lvl;
  if (ldexp(dt_soft, -lvl) > dt_des) *underflow = 1;
  if (lvl < prev_level - 1) lvl = prev_level - 1;
  while (lvl < OR_KMAX && (t_int & ((((int64_t)1) << (OR_KMAX - lvl)) - 1)) != 0) ++lvl;
  return lvl;
}

static double norm3(const double *v) {
  return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

/* First step of a member (Sec. 3.1): eta0 |a| / |j|. */
static double first_step(const double *a, const double *j, double eta0, double dt) {
  double jn = norm3(j);
  return jn > 0.0 ? eta0 * norm3(a) / jn : dt;
}

/* The hard acceleration (and jerk) of a composite is the mass-weighted mean  */
/* of its members' (Sec. 2.4.1): every evaluated member of a composite gets  */
/* sum_l m_l a_l / sum_l m_l, sums over the composite in ascending order.     */
static void average_sets(int64_t nc, const int64_t *set, const unsigned char *evald,
                         const double *m, double *a, double *jk) {
  for (int64_t r = 0; r < nc; ++r) {
    if (set[r] != r || !evald[r]) continue;
    int64_t size = 0;
    double M = 0.0, A[3] = {0, 0, 0}, J[3] = {0, 0, 0};
    for (int64_t l = 0; l < nc; ++l) {
      if (set[l] != r) continue;
      ++size;
      M += m[l];
      for (int c = 0; c < 3; ++c) { A[c] += m[l] * a[3 * l + c]; J[c] += m[l] * jk[3 * l + c]; }
    }
    if (size < 2) continue;
    for (int64_t l = 0; l < nc; ++l) {
      if (set[l] != r) continue;
      for (int c = 0; c < 3; ++c) { a[3 * l + c] = A[c] / M; jk[3 * l + c] = J[c] / M; }
    }
  }
}

/* Energy of the members marked in chg as far as a merge can change it:     */
/* their kinetic and star potential energy plus every pair potential with   */
/* at least one marked member (each pair once), pairs inside one composite  */
/* (set) left out.  Changeover functions replaced by unity.                 */
static double set_energy(int64_t nc, const unsigned char *chg, const int64_t *set,
                         const double *qx, const double *qy, const double *qz,
                         const double *qvx, const double *qvy, const double *qvz,
                         const double *m, const or_params *p) {
  double E = 0.0;
  for (int64_t k = 0; k < nc; ++k) {
    if (!chg[k]) continue;
    E += 0.5 * m[k] * (qvx[k] * qvx[k] + qvy[k] * qvy[k] + qvz[k] * qvz[k]);
    E -= p->G * p->m_star * m[k] / sqrt(qx[k] * qx[k] + qy[k] * qy[k] + qz[k] * qz[k]);
  }
  for (int64_t k = 0; k < nc; ++k) {
    if (!chg[k]) continue;
    for (int64_t l = 0; l < nc; ++l) {
      if (l == k || (chg[l] && l < k) || set[l] == set[k]) continue;
      double dx = qx[k] - qx[l], dy = qy[k] - qy[l], dz = qz[k] - qz[l];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      E -= p->G * m[k] * m[l] / sqrt(r2);
    }
  }
  return E;
}

/* Fourth-order Hermite with block individual time steps over [0, dt] for one */
/* cluster (Sec. 2.1.2, Makino 1991; Aarseth time steps).  Reading C7:        */
/*  predictor  x_p = x + v D + a D^2/2 + j D^3/6, v_p = v + a D + j D^2/2;    */
/*  corrector  a2 = (-6(a0-a1) - D(4 j0 + 2 j1))/D^2,                        */
/*             a3 = (12(a0-a1) + 6 D (j0 + j1))/D^3,                          */
/*             x = x_p + a2 D^4/24 + a3 D^5/120, v = v_p + a2 D^3/6 + a3 D^4/24;*/
/*  new step   sqrt(eta (|a||a2'| + |j|^2)/(|j||a3| + |a2'|^2)), a2' = a2+D a3;*/
/*  first step eta0 |a|/|j| (each hard step starts afresh, so every member's   */
/*  first step of the hard step uses eta0).  Everything in FP64, each formula  */
/*  evaluated as written, left to right.                                      */
/* All members are predicted to each block time; the active ones are        */
/* evaluated from the predicted state and then corrected together.           */
/*                                                                           */
/* Perfect accretion (Sec. 2.4.1), when RP (physical radii) is given         */
/* and f_radius > 0.  Readings:                                              */
/*  - detection: at every force evaluation (the initial one and each block   */
/*    time), each evaluated member k records its lowest-index partner j      */
/*    outside its composite with r_kj < f (R_p,k + R_p,j);                   */
/*  - after the correction, the members joined by these pairs (and the       */
/*    composites they already belong to) become one composite: each member   */
/*    is taken at the block time t_b (corrected if it was active, predicted  */
/*    otherwise), all get the centre-of-mass position and velocity, time t_b,*/
/*    the composite's hard acceleration and jerk (mass-weighted mean, pairs  */
/*    inside it left out) and a first step eta0 |a|/|j| (the paper's rule    */
/*    for the first step after a collision); the members stay separate       */
/*    particles until the merge after the second kick;                       */
/*  - dissipation (Eq. edisphard with the changeover functions replaced by   */
/*    unity, neighbours N_i taken as the cluster): the change of the energy  */
/*    of the affected members (kinetic, star potential, pair potential with  */
/*    the cluster) from before to after the replacement.                     */
/* root_out (nc entries, or NULL) receives for each member the lowest member */
/* of its composite (itself if none); *e_disp the dissipated energy;         */
/* msteps (nc entries, or NULL) the number of corrector steps of each member.*/
int or_hermite_cluster(int64_t nc, const int32_t *members, double *X, double *Y,
                       double *Z, double *VX, double *VY, double *VZ,
                       const double *M, const double *RO, const double *RPall,
                       const or_params *p, double dt, int64_t *n_steps,
                       int32_t *root_out, double *e_disp, int32_t *msteps) {
  if (msteps)
    for (int64_t k = 0; k < nc; ++k) msteps[k] = 0;
  const int64_t T = ((int64_t)1) << OR_KMAX;
  const double unit = ldexp(dt, -OR_KMAX);
  const int coll = RPall != NULL && p->f_radius > 0.0;
  double *buf = (double *)malloc(sizeof(double) * nc * 34);
  double *x = buf, *y = x + nc, *z = y + nc, *vx = z + nc, *vy = vx + nc, *vz = vy + nc;
  double *px = vz + nc, *py = px + nc, *pz = py + nc, *pvx = pz + nc, *pvy = pvx + nc, *pvz = pvy + nc;
  double *a = pvz + nc;   /* 3 nc */
  double *jk = a + 3 * nc; /* 3 nc */
  double *a1 = jk + 3 * nc, *j1 = a1 + 3 * nc;
  double *m = j1 + 3 * nc, *ro = m + nc, *rp = ro + nc;
  double *qx = rp + nc, *qy = qx + nc, *qz = qy + nc, *qvx = qz + nc, *qvy = qvx + nc,
         *qvz = qvy + nc; /* state at a collision's block time */
  int64_t *t = (int64_t *)malloc(sizeof(int64_t) * nc * 4);
  int64_t *set = t + nc, *oset = set + nc, *partner = oset + nc;
  int *lvl = (int *)malloc(sizeof(int) * nc);
  unsigned char *act = (unsigned char *)malloc(3 * nc);
  unsigned char *chg = act + nc, *croot = chg + nc;
  int underflow = 0;
  double edis = 0.0;
  for (int64_t k = 0; k < nc; ++k) {
    int32_t i = members[k];
    x[k] = X[i]; y[k] = Y[i]; z[k] = Z[i]; vx[k] = VX[i]; vy[k] = VY[i]; vz[k] = VZ[i];
    m[k] = M[i]; ro[k] = RO[i]; rp[k] = coll ? RPall[i] : 0.0;
    set[k] = k; partner[k] = -1; act[k] = 1;
  }
  const double *RP = coll ? rp : NULL;
  for (int64_t k = 0; k < nc; ++k)
    hard_acc_jerk_sets(nc, x, y, z, vx, vy, vz, m, ro, RP, set, p, k, a + 3 * k, jk + 3 * k,
                       &partner[k]);
  for (int64_t k = 0; k < nc; ++k) {
    t[k] = 0;
    lvl[k] = quantise_level(first_step(a + 3 * k, jk + 3 * k, p->eta0, dt), dt, 0, 0,
                            &underflow);
  }
  /* at t = 0 the block-time state is the initial state */
  memcpy(px, x, sizeof(double) * nc * 6);
  int64_t steps = 0, blocks = 0, tn = 0;
  int timeout = 0;
  for (;;) {
    /* a step below dt / 2^40 ends the cluster's integration (an error) */
    if (underflow) break;
    /* ---- collisions found by this evaluation (all members at tn) ---- */
    int any = 0;
    for (int64_t k = 0; k < nc; ++k) any |= partner[k] >= 0;
    if (any) {
      for (int64_t k = 0; k < nc; ++k) {
        const int on = act[k];
        qx[k] = on ? x[k] : px[k]; qy[k] = on ? y[k] : py[k]; qz[k] = on ? z[k] : pz[k];
        qvx[k] = on ? vx[k] : pvx[k]; qvy[k] = on ? vy[k] : pvy[k]; qvz[k] = on ? vz[k] : pvz[k];
        oset[k] = set[k];
      }
      for (int64_t k = 0; k < nc; ++k) {
        if (partner[k] < 0) continue;
        int64_t ra = set[k], rb = set[partner[k]];
        int64_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
        for (int64_t l = 0; l < nc; ++l) if (set[l] == hi) set[l] = lo;
      }
      for (int64_t k = 0; k < nc; ++k) croot[k] = 0;
      for (int64_t k = 0; k < nc; ++k) if (partner[k] >= 0) croot[set[k]] = 1;
      for (int64_t k = 0; k < nc; ++k) chg[k] = croot[set[k]];
      double Eb = set_energy(nc, chg, oset, qx, qy, qz, qvx, qvy, qvz, m, p);
      for (int64_t r = 0; r < nc; ++r) {
        if (!croot[r] || set[r] != r) continue;
        double Ms = 0.0, S[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t l = 0; l < nc; ++l) {
          if (set[l] != r) continue;
          Ms += m[l];
          S[0] += m[l] * qx[l]; S[1] += m[l] * qy[l]; S[2] += m[l] * qz[l];
          S[3] += m[l] * qvx[l]; S[4] += m[l] * qvy[l]; S[5] += m[l] * qvz[l];
        }
        for (int64_t l = 0; l < nc; ++l) {
          if (set[l] != r) continue;
          qx[l] = S[0] / Ms; qy[l] = S[1] / Ms; qz[l] = S[2] / Ms;
          qvx[l] = S[3] / Ms; qvy[l] = S[4] / Ms; qvz[l] = S[5] / Ms;
        }
      }
      double Ea = set_energy(nc, chg, set, qx, qy, qz, qvx, qvy, qvz, m, p);
      edis += Eb - Ea;
      for (int64_t k = 0; k < nc; ++k) {
        if (!chg[k]) continue;
        x[k] = qx[k]; y[k] = qy[k]; z[k] = qz[k];
        vx[k] = qvx[k]; vy[k] = qvy[k]; vz[k] = qvz[k];
        t[k] = tn;
      }
      for (int64_t k = 0; k < nc; ++k)
        if (chg[k])
          hard_acc_jerk_sets(nc, qx, qy, qz, qvx, qvy, qvz, m, ro, NULL, set, p, k,
                             a + 3 * k, jk + 3 * k, NULL);
      average_sets(nc, set, chg, m, a, jk);
      for (int64_t k = 0; k < nc; ++k) {
        if (!chg[k]) continue;
        lvl[k] = quantise_level(first_step(a + 3 * k, jk + 3 * k, p->eta0, dt), dt, 0, tn,
                                &underflow);
      }
      for (int64_t k = 0; k < nc; ++k) partner[k] = -1;
      if (underflow) break;
    }
    /* ---- next block time ---- */
    if (++blocks > OR_BLOCK_LIMIT) { timeout = 1; break; }
    tn = T;
    for (int64_t k = 0; k < nc; ++k) {
      int64_t e = t[k] + (T >> lvl[k]);
      if (e < tn) tn = e;
    }
    int64_t tmin = T;
    for (int64_t k = 0; k < nc; ++k) if (t[k] < tmin) tmin = t[k];
    if (tmin >= T) break;
    for (int64_t k = 0; k < nc; ++k) {
      /* predictor to the block time (reading C7) */
      double D = (double)(tn - t[k]) * unit;
      const double *ak = a + 3 * k, *jj = jk + 3 * k;
      double D2 = D * D, D3 = D2 * D;
      px[k] = x[k] + vx[k] * D + ak[0] * D2 / 2.0 + jj[0] * D3 / 6.0;
      py[k] = y[k] + vy[k] * D + ak[1] * D2 / 2.0 + jj[1] * D3 / 6.0;
      pz[k] = z[k] + vz[k] * D + ak[2] * D2 / 2.0 + jj[2] * D3 / 6.0;
      pvx[k] = vx[k] + ak[0] * D + jj[0] * D2 / 2.0;
      pvy[k] = vy[k] + ak[1] * D + jj[1] * D2 / 2.0;
      pvz[k] = vz[k] + ak[2] * D + jj[2] * D2 / 2.0;
      act[k] = (t[k] + (T >> lvl[k]) == tn);
    }
    for (int64_t k = 0; k < nc; ++k)
      if (act[k])
        hard_acc_jerk_sets(nc, px, py, pz, pvx, pvy, pvz, m, ro, RP, set, p, k, a1 + 3 * k,
                           j1 + 3 * k, &partner[k]);
    average_sets(nc, set, act, m, a1, j1);
    for (int64_t k = 0; k < nc; ++k) {
      if (!act[k]) continue;
      /* corrector (Makino & Aarseth 1992, reading C7) */
      double D = (double)(T >> lvl[k]) * unit;
      double D2 = D * D, D3 = D2 * D, D4 = D3 * D, D5 = D4 * D;
      double A2[3], A3[3], A2e[3];
      for (int c = 0; c < 3; ++c) {
        double a0 = a[3 * k + c], a1c = a1[3 * k + c];
        double j0 = jk[3 * k + c], j1c = j1[3 * k + c];
        A2[c] = (-6.0 * (a0 - a1c) - D * (4.0 * j0 + 2.0 * j1c)) / D2;
        A3[c] = (12.0 * (a0 - a1c) + 6.0 * D * (j0 + j1c)) / D3;
        A2e[c] = A2[c] + D * A3[c];  /* second derivative at the end of the step */
      }
      x[k] = px[k] + A2[0] * D4 / 24.0 + A3[0] * D5 / 120.0;
      y[k] = py[k] + A2[1] * D4 / 24.0 + A3[1] * D5 / 120.0;
      z[k] = pz[k] + A2[2] * D4 / 24.0 + A3[2] * D5 / 120.0;
      vx[k] = pvx[k] + A2[0] * D3 / 6.0 + A3[0] * D4 / 24.0;
      vy[k] = pvy[k] + A2[1] * D3 / 6.0 + A3[1] * D4 / 24.0;
      vz[k] = pvz[k] + A2[2] * D3 / 6.0 + A3[2] * D4 / 24.0;
      for (int c = 0; c < 3; ++c) { a[3 * k + c] = a1[3 * k + c]; jk[3 * k + c] = j1[3 * k + c]; }
      /* Aarseth step sqrt(eta (|a| |a2'| + |j|^2) / (|j| |a3| + |a2'|^2)) */
      double an = norm3(a + 3 * k), jn = norm3(jk + 3 * k);
      double a2n = norm3(A2e), a3n = norm3(A3);
      double num = an * a2n + jn * jn, den = jn * a3n + a2n * a2n;
      double dtd = den > 0.0 ? sqrt(p->eta * num / den) : dt;
      t[k] = tn;
      lvl[k] = quantise_level(dtd, dt, lvl[k], tn, &underflow);
      if (msteps) ++msteps[k];
      ++steps;
    }
  }
  for (int64_t k = 0; k < nc; ++k) {
    int32_t i = members[k];
    X[i] = x[k]; Y[i] = y[k]; Z[i] = z[k]; VX[i] = vx[k]; VY[i] = vy[k]; VZ[i] = vz[k];
    if (root_out) root_out[k] = (int32_t)set[k];
  }
  if (n_steps) *n_steps = steps;
  if (e_disp) *e_disp = edis;
  free(buf); free(t); free(lvl); free(act);
  if (timeout) return -5;
  return underflow ? -4 : 0;
}

/* ========================================================================= */
/* Kepler drift of isolated particles (Sec. 2.1.2: "solving the              */
/* Kepler equation with Newton-Raphson"; reading C9: mu = G M_*, no indirect  */
/* term).  Gauss f and g functions written with the change of eccentric      */
/* anomaly x = E - E0 (elliptic) or hyperbolic anomaly (hyperbolic):          */
/*   elliptic:  n dt = x - c sin x + s (1 - cos x),                           */
/*              c = 1 - r0/a, s = r0.v0 / sqrt(mu a);                         */
/*   hyperbolic (A = -a > 0): n dt = c sinh x + s (cosh x - 1) - x,           */
/*              c = 1 + r0/A, s = r0.v0 / sqrt(mu A).                         */
/* Returns -1 for an (unsupported) exactly parabolic orbit.                   */
/* ========================================================================= */
static int kepler_one(double *X, double *V, double dt, double mu) {
  double r0 = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  double v2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  double rv = X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
  double alpha = 2.0 / r0 - v2 / mu;
  double f, g, fd, gd;
  if (alpha > 0.0) {
    double a = 1.0 / alpha;
    double n = sqrt(mu / (a * a * a));
    double c = 1.0 - r0 / a, s = rv / sqrt(mu * a);
    /* strip whole orbits: f and g are periodic in x with period 2 pi */
    double P = 2.0 * M_PI / n;
    double k = floor(dt / P);
    double dtr = dt - k * P;
    double M = n * dtr;
    double xk = M;
    for (int it = 0; it < 100; ++it) {
      double F = xk - c * sin(xk) + s * (1.0 - cos(xk)) - M;
      double Fp = 1.0 - c * cos(xk) + s * sin(xk);
      double dx = F / Fp;
      xk -= dx;
      if (fabs(dx) <= 1e-15 * (1.0 + fabs(xk))) break;
    }
    double cx = cos(xk), sx = sin(xk);
    double r = a * (1.0 - c * cx + s * sx);
    f = 1.0 - (a / r0) * (1.0 - cx);
    g = dtr - (xk - sx) / n;
    fd = -sqrt(mu * a) * sx / (r * r0);
    gd = 1.0 - (a / r) * (1.0 - cx);
  } else if (alpha < 0.0) {
    double A = -1.0 / alpha;
    double n = sqrt(mu / (A * A * A));
    double c = 1.0 + r0 / A, s = rv / sqrt(mu * A);
    double M = n * dt;
    double xk = M * A / r0; /* first Newton iterate from the derivative at 0 */
    if (xk > 5.0) xk = log(2.0 * M / c + 1.0);
    for (int it = 0; it < 200; ++it) {
      double ch = cosh(xk), sh = sinh(xk);
      double F = c * sh + s * (ch - 1.0) - xk - M;
      double Fp = c * ch + s * sh - 1.0;
      double dx = F / Fp;
      if (dx > 1.0) dx = 1.0;
      if (dx < -1.0) dx = -1.0;
      xk -= dx;
      if (fabs(dx) <= 1e-15 * (1.0 + fabs(xk))) break;
    }
    double ch = cosh(xk), sh = sinh(xk);
    double r = A * (c * ch + s * sh - 1.0);
    f = 1.0 - (A / r0) * (ch - 1.0);
    g = dt - (sh - xk) / n;
    fd = -sqrt(mu * A) * sh / (r * r0);
    gd = 1.0 - (A / r) * (ch - 1.0);
  } else {
    return -1;
  }
  double nx[3], nv[3];
  for (int c = 0; c < 3; ++c) {
    nx[c] = f * X[c] + g * V[c];
    nv[c] = fd * X[c] + gd * V[c];
  }
  for (int c = 0; c < 3; ++c) { X[c] = nx[c]; V[c] = nv[c]; }
  return 0;
}

int or_kepler_drift(int64_t n, const int32_t *idx, double *x, double *y,
                    double *z, double *vx, double *vy, double *vz, double dt,
                    double mu) {
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t k = 0; k < n; ++k) {
    int64_t i = idx ? idx[k] : k;
    double X[3] = {x[i], y[i], z[i]}, V[3] = {vx[i], vy[i], vz[i]};
    if (kepler_one(X, V, dt, mu) != 0) { err |= 1; continue; }
    x[i] = X[0]; y[i] = X[1]; z[i] = X[2]; vx[i] = V[0]; vy[i] = V[1]; vz[i] = V[2];
  }
  return err ? -1 : 0;
}

/* Hard part of one soft step (procedure step 5): Hermite for every cluster   */
/* of >= 2 members, Kepler drift for isolated particles.                      */
int or_hard_step(int64_t n, double *x, double *y, double *z, double *vx,
                 double *vy, double *vz, const double *m, const double *r_out,
                 const double *RP, const or_params *p, double dt, int64_t n_single,
                 const int32_t *singles, int64_t n_clusters,
                 const int64_t *cl_off, const int32_t *cl_mem,
                 int64_t *n_hermite_steps, int32_t *comp_root, double *e_hard,
                 int32_t *member_steps) {
  int err = or_kepler_drift(n_single, singles, x, y, z, vx, vy, vz, dt, p->G * p->m_star);
  if (comp_root)
    for (int64_t i = 0; i < n; ++i) comp_root[i] = -1;
  if (member_steps)
    for (int64_t i = 0; i < n; ++i) member_steps[i] = 0;
  double *ec = (double *)calloc(n_clusters > 0 ? n_clusters : 1, sizeof(double));
  int64_t steps = 0;
  int herr = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : steps) reduction(min : herr)
  for (int64_t c = 0; c < n_clusters; ++c) {
    int64_t ns = 0;
    const int64_t nc = cl_off[c + 1] - cl_off[c];
    const int32_t *mem = cl_mem + cl_off[c];
    int32_t *root = (int32_t *)malloc(sizeof(int32_t) * 3 * nc);
    int32_t *cnt = root + nc, *ms = cnt + nc;
    int e = or_hermite_cluster(nc, mem, x, y, z, vx, vy, vz, m, r_out, RP, p, dt, &ns, root,
                               &ec[c], ms);
    if (member_steps)
      for (int64_t k = 0; k < nc; ++k) member_steps[mem[k]] = ms[k];
    if (comp_root) {
      /* members of composites of two or more: the caller index of the lowest */
      for (int64_t k = 0; k < nc; ++k) cnt[k] = 0;
      for (int64_t k = 0; k < nc; ++k) ++cnt[root[k]];
      for (int64_t k = 0; k < nc; ++k)
        if (cnt[root[k]] >= 2) comp_root[mem[k]] = mem[root[k]];
    }
    free(root);
    if (e) herr = e;
    steps += ns;
  }
  double et = 0.0;
  for (int64_t c = 0; c < n_clusters; ++c) et += ec[c];
  free(ec);
  if (e_hard) *e_hard = et;
  if (n_hermite_steps) *n_hermite_steps = steps;
  if (err) return -1;
  return herr;
}

/* ========================================================================= */
/* Second kick of composites and the merge (Sec. 2.4.1).                     */
/* After the soft force of procedure step 7, the members of a composite are  */
/* kicked with the mass-weighted mean of their soft accelerations,           */
/*   a_c = sum_l m_l a_l / sum_l m_l (ascending l),                           */
/* every other particle with its own.  The dissipation is the relative       */
/* kinetic energy the separate kicks would have given: per composite         */
/*   sum_l m_l |h (a_l - a_c)|^2 / 2,                                         */
/* summed over composites in ascending order of their lowest member.         */
/* comp_root[i]: lowest member of i's composite, or -1.                      */
/* ========================================================================= */
static int64_t composite_list(int64_t n, const int32_t *comp_root, int32_t **list) {
  int64_t nl = 0;
  for (int64_t i = 0; i < n; ++i) nl += comp_root[i] >= 0;
  *list = (int32_t *)malloc(sizeof(int32_t) * (nl > 0 ? nl : 1));
  nl = 0;
  for (int64_t i = 0; i < n; ++i)
    if (comp_root[i] >= 0) (*list)[nl++] = (int32_t)i;
  return nl;
}

double or_kick_composites(int64_t n, double *vx, double *vy, double *vz,
                          const double *ax, const double *ay, const double *az,
                          double h, const double *m, const int32_t *comp_root) {
  for (int64_t i = 0; i < n; ++i) {
    if (comp_root[i] >= 0) continue;
    vx[i] += ax[i] * h; vy[i] += ay[i] * h; vz[i] += az[i] * h;
  }
  int32_t *list;
  int64_t nl = composite_list(n, comp_root, &list);
  double E = 0.0;
  for (int64_t q = 0; q < nl; ++q) {
    const int32_t r = list[q];
    if (comp_root[r] != r) continue;
    double M = 0.0, A[3] = {0, 0, 0};
    for (int64_t u = 0; u < nl; ++u) {
      const int32_t l = list[u];
      if (comp_root[l] != r) continue;
      M += m[l];
      A[0] += m[l] * ax[l]; A[1] += m[l] * ay[l]; A[2] += m[l] * az[l];
    }
    const double ac[3] = {A[0] / M, A[1] / M, A[2] / M};
    double Es = 0.0;
    for (int64_t u = 0; u < nl; ++u) {
      const int32_t l = list[u];
      if (comp_root[l] != r) continue;
      vx[l] += ac[0] * h; vy[l] += ac[1] * h; vz[l] += ac[2] * h;
      const double dx = (ax[l] - ac[0]) * h, dy = (ay[l] - ac[1]) * h, dz = (az[l] - ac[2]) * h;
      Es += 0.5 * m[l] * (dx * dx + dy * dy + dz * dz);
    }
    E += Es;
  }
  free(list);
  return E;
}

/* Procedure step 9: each composite becomes one particle at its lowest index:*/
/* mass sum_l m_l, physical radius (sum_l R_l^3)^(1/3) (reading: volume is   */
/* kept, all bodies having one density), position and velocity those of its */
/* members (identical after the kick above).  The other members are removed */
/* and the survivors keep their order: new_index[i] = i's new index or -1.   */
/* Returns the new particle count.  r_out and r_search are carried along;    */
/* the caller recomputes them (and the soft force) afterwards.               */
int64_t or_merge(int64_t n, double *x, double *y, double *z, double *vx, double *vy,
                 double *vz, double *m, double *rp, double *r_out, double *r_search,
                 const int32_t *comp_root, int32_t *new_index) {
  int32_t *list;
  int64_t nl = composite_list(n, comp_root, &list);
  for (int64_t q = 0; q < nl; ++q) {
    const int32_t r = list[q];
    if (comp_root[r] != r) continue;
    double M = 0.0, V = 0.0;
    for (int64_t u = 0; u < nl; ++u) {
      const int32_t l = list[u];
      if (comp_root[l] != r) continue;
      M += m[l];
      V += rp[l] * rp[l] * rp[l];
    }
    m[r] = M;
    rp[r] = cbrt(V);
  }
  free(list);
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (comp_root[i] >= 0 && comp_root[i] != i) { new_index[i] = -1; continue; }
    new_index[i] = (int32_t)k;
    x[k] = x[i]; y[k] = y[i]; z[k] = z[i]; vx[k] = vx[i]; vy[k] = vy[i]; vz[k] = vz[i];
    m[k] = m[i]; rp[k] = rp[i]; r_out[k] = r_out[i]; r_search[k] = r_search[i];
    ++k;
  }
  return k;
}

/* ========================================================================= */
/* Total energy.  H_soft + H_hard (Eqs. soft, hard) with                    */
/* W + (1 - W) = 1 is the Newtonian energy                                    */
/*   E = sum m v^2 / 2 - sum G M_* m / r - sum_{i<j} G m_i m_j / r_ij.        */
/* out = {E, kinetic, star potential, pair potential}.                       */
/* ========================================================================= */
void or_energy(int64_t n, const double *x, const double *y, const double *z,
               const double *vx, const double *vy, const double *vz,
               const double *m, double G, double m_star, double out[4]) {
  double ek = 0.0, es = 0.0, ep = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : ek, es, ep)
  for (int64_t i = 0; i < n; ++i) {
    ek += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
    es -= G * m_star * m[i] / sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    double s = 0.0;
    for (int64_t j = i + 1; j < n; ++j) {
      double rx = x[i] - x[j], ry = y[i] - y[j], rz = z[i] - z[j];
      s += m[j] / sqrt(rx * rx + ry * ry + rz * rz);
    }
    ep -= G * m[i] * s;
  }
  out[0] = ek + es + ep; out[1] = ek; out[2] = es; out[3] = ep;
}
