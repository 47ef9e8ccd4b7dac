// Internal definitions of the GB300 adaptive MR-LBM library: geometry and
// scheme constants, Morton keys with a root prefix, the dense per-level
// index space, the device mesh layout and the kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MR_MAXL 16       // levels 0..15
#define MR_MAXQ 16       // populations per cell
#define MR_DENSE_ALIGN 1024u

// cell classes stored in the two top bits of an index-map entry
#define MR_CLS_LEAF 0u
#define MR_CLS_INT 1u
#define MR_CLS_GHOST 2u
#define MR_MAP_NONE (-1)

// adaptation flags (dense byte per cell of levels J_min..J-1)
#define MR_F_T 1u   // children kept by T_eps (with closure)
#define MR_F_H 2u   // refined after H_eps
#define MR_F_G 4u   // refined by the grading
// classification (dense byte per cell of levels J_min..J)
#define MR_C_LEAF 1u
#define MR_C_INT 2u
#define MR_C_GHOST 4u
#define MR_C_INPUT 8u
#define MR_C_STEN 16u  // ghost marking: the prediction stencil around this cell is claimed

// device error bits
#define MR_DERR_CAPACITY 1
#define MR_DERR_INTERNAL 2
#define MR_DERR_NONFINITE 4
#define MR_DERR_INPUT 8

// weight tables: [level][axis][slot][table][5], table 0: (R_{k-1} - R_k),
// 1: (L_{k+1} - L_k), 2: R_k, 3: L_k, delta = -2..2.
#define MR_NSLOT 5
#define MR_NTAB 4
#define MR_WIDX(l, a, s, t) (((((l) * 3 + (a)) * MR_NSLOT + (s)) * MR_NTAB + (t)) * 5)

struct Geo {
  int scheme, d, q, m, Q, ncons;
  int Jmin, J;
  int roots[3];
  int n[MR_MAXL][3];           // cells per axis at each level
  uint32_t ncode[MR_MAXL];     // valid codes per level (= cells)
  uint32_t base[MR_MAXL + 1];  // dense base index of each level, aligned; base[J+1] = dense size
  int periodic[3];
  int bc[6];
  double lambda;
  double inv_lambda;
  double s[16];
  double phys[8];
  double eps;
  int mu_bar;
  int cross_sign;
  int eta[9][3];
  int opp[9];
  int cap[3];                  // capacities: leaf, internal, ghost
  double consw[4][MR_MAXQ];    // conserved moments as linear forms of the populations
  int form;                    // storage / compute form, see MR_FORM_*
  double off[MR_MAXQ];         // stored value = population - off[p] (0 unless 16-bit storage)
  int s_pred;                  // half-width s of the prediction operator (Table 1): 1, 2 or 3
  int diag;                    // lattice with diagonal velocities: 5^d stream window
  int obstacle;                // penalisation of Sec. 7.2.2 after the collision
  double obs[3];               // obstacle disc: centre x, y and radius
  double xlo[2];               // domain origin
  double dxJ;                  // finest cell size
  double feq0[MR_MAXQ];        // equilibrium populations at (rho0, 0, 0)
  double bcv[MR_MAXQ];         // f^{h,eq} - f^{h dagger,eq} at (rho0, u0): bounce back with velocity
  // FP32 copies of the constants used by FP32 arithmetic (no per-cell conversion)
  struct {
    float lambda, inv_lambda, cross_sign;
    float s[16], phys[8], off[MR_MAXQ], feq0[MR_MAXQ], bcv[MR_MAXQ];
  } f32;
};

// Storage / compute forms: populations are stored as S and transported and
// collided in C; details (the mesh decisions) are always evaluated in FP64.
#define MR_FORM_F64 0        // S = double, C = double (plain)
#define MR_FORM_F32 1        // S = float,  C = float
#define MR_FORM_F32_F16 2    // S = half (offset from the rest equilibrium), C = float
#define MR_FORM_F32_BF16 3   // S = bfloat16 (offset from the rest equilibrium), C = float

// counters of one mesh, in device memory
struct MeshCounts {
  int total[3];                 // leaves, internal, ghosts
  int off[3][MR_MAXL + 1];      // offsets of each level in the class arrays
  int err;                      // device error bits
  int pad;
  long long leaf_updates;       // sum of leaf counts over steps
  long long steps;
};

struct MeshDev {
  uint32_t* code[3];   // Morton code (with root prefix) at own level
  uint8_t* lvl[3];
  int32_t* map;        // dense index map: (cls << 30) | idx, or -1
  void* IF;            // internal-cell values [Q][cap_int], storage type of the form
  void* GF;            // ghost values [Q][cap_ghost], storage type of the form
  double* G;           // group norm per internal cell
  int32_t* src;        // per leaf: source entry in the previous mesh, -1 if predicted
  MeshCounts* cnt;
  uint8_t* mact;       // per dense chunk: 1 if map holds an entry (not -1) in it
};

// ------------------------------------------------------------------------
// Morton keys with root prefix
// ------------------------------------------------------------------------

__host__ __device__ inline uint32_t mr_spread2(uint32_t x) {
  x &= 0x0000FFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__host__ __device__ inline uint32_t mr_compact2(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}

// three-way interleave of 10-bit integers (d = 3)
__host__ __device__ inline uint32_t mr_spread3(uint32_t x) {
  x &= 0x000003FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}
__host__ __device__ inline uint32_t mr_compact3(uint32_t x) {
  x &= 0x09249249u;
  x = (x | (x >> 2)) & 0x030C30C3u;
  x = (x | (x >> 4)) & 0x0300F00Fu;
  x = (x | (x >> 8)) & 0x030000FFu;
  x = (x | (x >> 16)) & 0x000003FFu;
  return x;
}

__host__ __device__ inline uint32_t mr_encode(const Geo& g, int l, int x, int y) {
  if (g.d == 1) return (uint32_t)x;
  uint32_t mask = (1u << l) - 1u;
  uint32_t root = (uint32_t)(x >> l) + (uint32_t)g.roots[0] * (uint32_t)(y >> l);
  uint32_t local = mr_spread2((uint32_t)x & mask) | (mr_spread2((uint32_t)y & mask) << 1);
  return (root << (2 * l)) | local;
}

__host__ __device__ inline void mr_decode(const Geo& g, int l, uint32_t code, int& x, int& y) {
  if (g.d == 1) {
    x = (int)code;
    y = 0;
    return;
  }
  uint32_t root = code >> (2 * l);
  uint32_t local = code & ((l > 0) ? ((1u << (2 * l)) - 1u) : 0u);
  int rx = (int)(root % (uint32_t)g.roots[0]), ry = (int)(root / (uint32_t)g.roots[0]);
  x = (rx << l) | (int)mr_compact2(local);
  y = (ry << l) | (int)mr_compact2(local >> 1);
}

// d = 3: (root << 3l) | spread3(x) | spread3(y) << 1 | spread3(z) << 2, with
// root = x >> l + roots_x (y >> l + roots_y (z >> l))
__host__ __device__ inline uint32_t mr_encode3(const Geo& g, int l, int x, int y, int z) {
  uint32_t mask = (1u << l) - 1u;
  uint32_t root = (uint32_t)(x >> l) +
                  (uint32_t)g.roots[0] * ((uint32_t)(y >> l) + (uint32_t)g.roots[1] * (uint32_t)(z >> l));
  uint32_t local = mr_spread3((uint32_t)x & mask) | (mr_spread3((uint32_t)y & mask) << 1) |
                   (mr_spread3((uint32_t)z & mask) << 2);
  return (root << (3 * l)) | local;
}
__host__ __device__ inline void mr_decode3(const Geo& g, int l, uint32_t code, int& x, int& y, int& z) {
  uint32_t root = code >> (3 * l);
  uint32_t local = code & ((l > 0) ? ((1u << (3 * l)) - 1u) : 0u);
  const uint32_t rxy = (uint32_t)g.roots[0] * (uint32_t)g.roots[1];
  int rz = (int)(root / rxy), rr = (int)(root % rxy);
  int rx = rr % g.roots[0], ry = rr / g.roots[0];
  x = (rx << l) | (int)mr_compact3(local);
  y = (ry << l) | (int)mr_compact3(local >> 1);
  z = (rz << l) | (int)mr_compact3(local >> 2);
}

// periodic wrap of a cell index a few cells outside [0, n): every caller
// steps at most two cells from a cell inside, so each loop runs at most a
// few times (short code instead of an integer division)
__host__ __device__ inline int mr_wrap(int x, int n) {
  while (x < 0) x += n;
  while (x >= n) x -= n;
  return x;
}

// neighbour for the mesh rules: periodic wrap, false outside the domain
__host__ __device__ inline bool mr_nbr_mesh(const Geo& g, int l, int& x, int& y) {
  int nx = g.n[l][0], ny = g.n[l][1];
  if (x < 0 || x >= nx) {
    if (!g.periodic[0]) return false;
    x = mr_wrap(x, nx);
  }
  if (g.d >= 2 && (y < 0 || y >= ny)) {
    if (!g.periodic[1]) return false;
    y = mr_wrap(y, ny);
  }
  if (g.d == 1) y = 0;
  return true;
}

// stencil cell of the prediction operator: periodic wrap, otherwise the
// nearest cell of the same level (constant extension)
__host__ __device__ inline void mr_nbr_stencil(const Geo& g, int l, int& x, int& y) {
  int nx = g.n[l][0], ny = g.n[l][1];
  if (x < 0 || x >= nx) x = g.periodic[0] ? mr_wrap(x, nx) : (x < 0 ? 0 : nx - 1);
  if (g.d >= 2) {
    if (y < 0 || y >= ny) y = g.periodic[1] ? mr_wrap(y, ny) : (y < 0 ? 0 : ny - 1);
  } else {
    y = 0;
  }
}

// Dimension-generic forms of the above on a coordinate array c[D]: for D <= 2
// they call the two-coordinate functions (c[1] = 0 when D = 1).
template <int D>
__host__ __device__ inline uint32_t mr_encode_d(const Geo& g, int l, const int* c) {
  if constexpr (D == 3)
    return mr_encode3(g, l, c[0], c[1], c[2]);
  else
    return mr_encode(g, l, c[0], D == 2 ? c[1] : 0);
}
template <int D>
__host__ __device__ inline void mr_decode_d(const Geo& g, int l, uint32_t code, int* c) {
  if constexpr (D == 3) {
    mr_decode3(g, l, code, c[0], c[1], c[2]);
  } else {
    int x, y;
    mr_decode(g, l, code, x, y);
    c[0] = x;
    if (D == 2) c[1] = y;
  }
}
template <int D>
__host__ __device__ inline bool mr_nbr_mesh_d(const Geo& g, int l, int* c) {
  for (int a = 0; a < D; ++a) {
    const int n = g.n[l][a];
    if (c[a] < 0 || c[a] >= n) {
      if (!g.periodic[a]) return false;
      c[a] = mr_wrap(c[a], n);
    }
  }
  return true;
}
template <int D>
__host__ __device__ inline void mr_nbr_stencil_d(const Geo& g, int l, int* c) {
  for (int a = 0; a < D; ++a) {
    const int n = g.n[l][a];
    if (c[a] < 0 || c[a] >= n) c[a] = g.periodic[a] ? mr_wrap(c[a], n) : (c[a] < 0 ? 0 : n - 1);
  }
}
// 3^D stencil / 2^D children counts
template <int D>
struct Pow3 {
  static constexpr int value = D == 1 ? 3 : D == 2 ? 9 : 27;
};

__host__ __device__ inline int mr_slot(int k, int N, int periodic) {
  if (periodic) return 2;
  if (k < 2) return k;
  if (k >= N - 2) return 3 + (k - (N - 2));
  return 2;
}

// Flattened weights of the prediction of half-width s = 2, 3: the window is
// W = 2s cells on either side, so a table has 2W + 1 entries, and 2W + 1
// slots tell apart the cells within W of a non-periodic face (a level of
// at most 2W + 1 cells gets one slot per cell).
// Layout: [level][axis][slot 0..2W][table 0..3][2W + 1], tables as above.
#define MR_WWIDX(l, a, sl, t, W) (((((l) * 3 + (a)) * (2 * (W) + 1) + (sl)) * MR_NTAB + (t)) * (2 * (W) + 1))
__host__ __device__ inline int mr_slot_w(int k, int N, int periodic, int W) {
  if (periodic) return W;
  if (N <= 2 * W + 1) return k;
  if (k < W) return k;
  if (k >= N - W) return W + 1 + (k - (N - W));
  return W;
}

// ------------------------------------------------------------------------
// instances and groups
// ------------------------------------------------------------------------

#define MR_MAXB 1024  // instances of one group

// Everything the step kernels need about one instance, in device memory.
// Leaf-value arrays are void*: their element type is the storage type of
// g.form.  fstate holds the stored (post-collision) leaf values of the
// current mesh, fscratch the values moved to the new mesh before transport.
struct __align__(16) InstDev {
  Geo g;
  MeshDev mesh[2];
  void* fstate;
  void* fscratch;
  uint8_t* flags;     // dense: T / H / G marks
  uint8_t* cls;       // dense: classification of the new mesh
  uint8_t* act;       // per dense chunk: 1 if a cell of it may be flagged, in the new tree or a ghost
  uint8_t* acth;      // per dense chunk: 1 if a cell of it may carry the H flag (grading seeds)
  int* bcounts;       // per dense chunk: leaf / internal / ghost counts, then offsets
  const double* W;    // flattened weights, MR_WIDX layout
  const float* Wf;    // the same in FP32
  void* det;          // D2Q9 with s = 1, and every scheme with s = 2, 3: the children's details of
                      // the refined cells that leaves reach with their transport windows,
                      // [(child * Q + p) * cap_int + internal index] in the form's arithmetic type
  const double* Ws;   // s = 2, 3: flattened weights of half-width 2s, MR_WWIDX layout (else null)
  const float* Wsf;   // the same in FP32
};

// Launch schedule of a group: for each phase, the blocks per SM its tiled
// kernels may use (the grid is at most nsm times that; blocks stride over
// the tiles).  Defaults below; mr_lbm_batch_autotune picks them per group.
enum { MR_PH_PROJECT = 0, MR_PH_DETAILS, MR_PH_FLAGS, MR_PH_COMPACT, MR_PH_REMESH, MR_PH_PREDICT, MR_PH_STREAM,
       MR_NPH };
#define MR_DEFAULT_BPS {8, 8, 4, 8, 8, 8, 8}

// Instances of one scheme and storage form, stepped by shared launches: every
// step kernel covers all of them (a single solver is a group of one).  All
// instances of a group are on the same mesh parity.
struct Group {
  const InstDev* dev;    // device array [n]
  const int* chunk_pre;  // device array [n + 1]: first dense chunk of each instance
  int n;
  int d, Q, scheme, form;
  int s;                 // half-width of the prediction (all instances alike)
  int bps[MR_NPH];       // launch schedule: blocks per SM of each phase
  int chunks;            // dense chunks of all instances
  int span;              // maximum of J - J_min
  bool grade;            // some instance has J > J_min + 1
  long long capL, capI;  // summed leaf / internal capacities
  long long proj_cells[MR_MAXL];  // summed cells of level J - k (projection phase k)
  long long pred_cells[MR_MAXL];  // summed cells of level J_min + k (prediction phase k)
  int nsm;
  // the original adaptive collision (a group of one only): dense FP64
  // reconstruction buffer [Q][exact_nd] indexed like the dense map, or null
  double* exact = nullptr;
  long long exact_nd = 0;
};

// Launch of a step kernel with programmatic dependent launch: the next
// kernel of the stream may be scheduled while this one drains.  Every
// kernel launched this way calls mr_grid_dep(), which waits for the grid
// before it to complete and its writes to be visible, before it reads
// anything an earlier kernel writes (only the copy of its instance
// descriptor, written by the host before the step, comes first), so the
// order of the stream is kept; only the launch latency is overlapped.
template <typename... KArgs, typename... Args>
inline cudaError_t mr_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Grid of a tiled step kernel: at most `per_sm` blocks per SM, and no more
// blocks than the tiles the group can have for `max_items` items.
inline int mr_tile_grid(const Group& G, long long max_items, int items_per_tile, int per_sm) {
  const long long need = (max_items + items_per_tile - 1) / items_per_tile + G.n;
  const long long cap = (long long)G.nsm * per_sm;
  return (int)(need < cap ? need : cap);
}
// dynamic shared memory of a tiled step kernel: the tile prefix
inline size_t mr_pre_bytes(const Group& G) { return (size_t)(G.n + 1) * sizeof(int); }

// ------------------------------------------------------------------------
// kernels (defined in mr_encode.cu, mr_mesh.cu, mr_stream.cu)
// ------------------------------------------------------------------------

// Step kernels, one launch for every instance of a group.  `cur` is the
// parity of the current mesh (values in fstate); the new mesh is 1 - cur.
void mr_launch_project(const Group& G, int cur, int k, cudaStream_t st);  // level J - k
void mr_launch_details(const Group& G, int cur, cudaStream_t st);
void mr_launch_flags_T(const Group& G, int cur, cudaStream_t st);
void mr_launch_flags_H(const Group& G, int cur, cudaStream_t st);
void mr_launch_grade(const Group& G, cudaStream_t st);
void mr_launch_classify(const Group& G, cudaStream_t st);
void mr_launch_mark_ghosts(const Group& G, cudaStream_t st);
int mr_chunk_blocks_grid(const Group& G);  // grid of the dense kernels that take a block per chunk
void mr_launch_compact(const Group& G, int dst, cudaStream_t st);  // count + scan + scatter into mesh dst
void mr_launch_remesh_copy(const Group& G, int cur, cudaStream_t st);
void mr_launch_predict_level(const Group& G, int dst, int k, cudaStream_t st);  // level J_min + k
// D2Q9, s = 1: the details of the children of every refined cell of mesh dst
// that a leaf of its own level borders, for the transport's critical case.
void mr_launch_edge_details(const Group& G, int dst, cudaStream_t st);
// count = 1: also add the step to the instances' counters (once per step)
void mr_launch_stream_collide(const Group& G, int dst, int do_stream, int do_collide, cudaStream_t st,
                              int count = 0);
// Original adaptive collision of the post-transport leaves of mesh dst
// (mr_exact.cu); returns the number of launches.
int mr_launch_exact_collision(const Group& G, int dst, double* Fd, long long nd, cudaStream_t st);

// Input / output kernels of one instance.
void mr_launch_init_eq(const Geo& g, const MeshDev& B, const double* cons, void* LF,
                       cudaStream_t st, int grid);
void mr_launch_full_mesh(const Geo& g, uint8_t* cls, uint8_t* act, cudaStream_t st, int grid);
void mr_launch_leaves_in(const Geo& g, long long n, const unsigned long long* keys,
                         const signed char* levels, int32_t* inidx, uint8_t* cls, uint8_t* act, MeshCounts* cnt,
                         unsigned long long* vol, cudaStream_t st, int grid);
void mr_launch_leaves_check(const Geo& g, uint8_t* cls, MeshCounts* cnt, cudaStream_t st, int grid);
void mr_launch_gather_input(const Geo& g, const MeshDev& B, const int32_t* inidx, long long n,
                            const double* fin, void* LF, cudaStream_t st, int grid);
void mr_launch_leaves_out(const Geo& g, const MeshDev& B, const void* LF, long long n,
                          unsigned long long* keys, signed char* levels, double* f,
                          cudaStream_t st, int grid);
void mr_launch_project_dense(const Geo& g, const MeshDev& B, const void* LF, int level,
                             const double* prev, double* cur, cudaStream_t st, int grid);
size_t mr_form_bytes(int form);  // bytes per stored population value

// The same phases for the prediction of half-width s = 2, 3 (mr_wide.cu):
// (2s+1)^d stencils, grading and ghost cascades of radius s, transport
// windows of 2s cells on either side.  The launchers above call these when
// the group's s is above 1.
void mr_launch_details_w(const Group& G, int cur, cudaStream_t st);
void mr_launch_grade_w(const Group& G, cudaStream_t st);
void mr_launch_mark_ghosts_w(const Group& G, cudaStream_t st);
void mr_launch_predict_level_w(const Group& G, int dst, int k, cudaStream_t st);
void mr_launch_edge_details_w(const Group& G, int dst, cudaStream_t st);  // before the wide transport
void mr_launch_stream_collide_w(const Group& G, int dst, int do_stream, int do_collide, cudaStream_t st, int count);
void mr_launch_project_dense_w(const Geo& g, const MeshDev& B, const void* LF, int level, const double* prev,
                               double* cur, cudaStream_t st, int grid);

// Adjoint kernels (mr_adjoint.cu), FP64, one instance; A = mesh of step n,
// B = mesh of step n + 1, adjoint arrays in the layout of the value arrays.
void mr_adj_collide(const Geo& g, const MeshDev& B, const double* z, double* lam, double* ds, int source,
                    double vol_J, cudaStream_t st, int grid);
void mr_adj_transport(const Geo& g, const MeshDev& B, const double* W, const double* mu, double* aL, double* aI,
                      double* aG, cudaStream_t st, int grid);
void mr_adj_predict(const Geo& g, const MeshDev& B, int level, double* aL, double* aI, double* aG, cudaStream_t st,
                    int grid);
void mr_adj_transfer(const Geo& g, const MeshDev& A, const MeshDev& B, const double* aLB, const double* aIB,
                     double* aLA, double* aIA, cudaStream_t st, int grid);
void mr_adj_project(const Geo& g, const MeshDev& A, int level, double* aLA, double* aIA, cudaStream_t st, int grid);
void mr_adj_init(const Geo& g, const MeshDev& B, const double* cons, const double* lam, double* grad,
                 cudaStream_t st, int grid);
void mr_kinetic_energy(const Geo& g, const MeshDev& B, const double* LF, double vol_J, double* J, cudaStream_t st,
                       int grid);
