/*
 * Plain FP64 CPU oracle of the fully adaptive multiresolution lattice-Boltzmann
 * step (Bellotti, Gouarin, Graille, Massot, arXiv 2103.02903).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: it exists so that the tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against a slow, dense,
 * literal restatement of the paper.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Data layout: every level l in [J_min, J] is a dense row-major array of
 * N_l = roots_x 2^l (x) roots_y 2^l (y) roots_z 2^l (z) cells, x fastest.
 * Populations are stored per cell, Q contiguous doubles (Q = q * m for
 * vectorial schemes, lattice-major).
 */
#ifndef MR_ORACLE_H
#define MR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_D1Q2_ADVECTION = 0,
  OR_D1Q2_BURGERS = 1,
  OR_D1Q3_SHALLOW_WATER = 2,
  OR_D2Q4x4_EULER = 3,
  OR_D2Q9_NS = 4,
  OR_D3Q6_ADVECTION = 5
};

enum { OR_BC_PERIODIC = 0, OR_BC_COPY = 1, OR_BC_BOUNCE_BACK = 2,
       OR_BC_ANTI_BOUNCE_BACK = 3, OR_BC_BOUNCE_BACK_VELOCITY = 4 };

typedef struct {
  int scheme;
  double lambda;       /* lattice velocity, Eq. acousticscaling */
  double s[16];        /* relaxation rates of the non-conserved moments */
  double phys[8];      /* scheme constants: V | g | gamma | rho0,u0x,u0y,cx,cy,r */
  double xmin[3], xmax[3];
  int roots[3];        /* cells per axis at level 0 */
  int min_level, max_level;
  double eps;          /* threshold epsilon of Eq. Thresholding */
  int mu_bar;          /* regularity guess of the refinement rule, in [0, 2s + 1] (Sec. 5.1);
                          or_create refuses other values */
  int bc[6];           /* -x,+x,-y,+y,-z,+z */
  int cross_sign;      /* +1 tensor-product prediction, -1 diagonal term as printed */
  int obstacle;        /* 1: volume-fraction penalisation after collision (Sec. 7.2) */
  int exact_collision; /* 1: collide the reconstructed finest data, then average (Eq. sourceoferror) */
  int pred_s;          /* prediction stencil half-width s = 1, 2, 3 (Table 1); 0 reads as 1 */
} or_config;

typedef struct or_state or_state;

or_state* or_create(const or_config* cfg);
void or_destroy(or_state* st);
int or_scheme_info(const or_state* st, int* d, int* q, int* m, int* Q, int* ncons);

/* Algorithm 1 initialisation: full finest mesh at equilibrium of the given
 * level-J conserved moments, SoA [ncons][N_J]. */
int or_init(or_state* st, const double* conserved);
/* One or more full time steps: adapt (T, H, G), remesh, stream, collide. */
int or_step(or_state* st, int nsteps);
/* Mesh adaptation and remesh only (no stream / collide). */
int or_adapt(or_state* st);
/* Stream and collide on the current mesh (no adaptation). */
int or_stream_collide(or_state* st, int do_collide);

long long or_num_leaves(const or_state* st);
/* Leaves sorted by (level, z, y, x); f is SoA [Q][n]. */
int or_get_leaves(const or_state* st, int* level, int* ix, int* iy, int* iz, double* f);
/* Replace the state by the given leaves (must partition the domain). */
int or_set_leaves(or_state* st, long long n, const int* level, const int* ix,
                  const int* iy, const int* iz, const double* f);
/* Conserved moments of the reconstructed field on uniform level `level`,
 * SoA [ncons][N_level] row-major. */
int or_project(or_state* st, int level, double* out);
/* Population field reconstructed on uniform level `level`, SoA [Q][N_level]. */
int or_reconstruct(or_state* st, int level, double* out);
/* Smallest relative distance of a group norm to a threshold in the last
 * adaptation (Eq. Thresholding and the refinement rule). */
double or_last_margin(const or_state* st);
/* Group norms of the last adaptation, dense level `level` (parents),
 * -1 where the cell was not an internal cell. */
int or_group_norms(const or_state* st, int level, double* out);

/* Raw operators for the pins. */
double or_prediction_coefficient(void);
/* Predict the 2^d children of a level-0 parent from a (3)^d stencil given
 * row-major (x fastest); out[ci] with ci = dx + 2 dy + 4 dz. */
int or_predict_children(int d, int cross_sign, const double* stencil, double* out);
/* Table 1 coefficients c_1 .. c_s of the prediction of half-width s (1..3). */
int or_prediction_coefficients(int s, double* out);
/* The prediction of half-width s on a (2s+1)^d stencil (x fastest): the 2^d
 * children's values, child index (dz << 2) | (dy << 1) | dx. */
int or_predict_children_s(int d, int cross_sign, int s, const double* stencil, double* out);
/* Mesh invariants of the current state: 1 if the leaves form a graded tree. */
int or_check_graded(const or_state* st);

#ifdef __cplusplus
}
#endif
#endif
