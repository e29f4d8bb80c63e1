/*
 * FP64 CPU oracle of the two-pass MBOIT puzzle-piece render.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no source with the CUDA path.
 *
 * Coordinates follow the `scenes` module: field[z][y][x] float32 vertex
 * values, vertex (x,y,z) at point (x,y,z), bricks of 2^brick_log2 cells,
 * brick id (bz*nby + by)*nbx + bx.
 */
#ifndef MBOIT_ORACLE_H
#define MBOIT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float eye[3], u[3], v[3], w[3];
    int32_t width, height, projection, reserved;
    float scale_u, scale_v, znear, zfar;
} orc_view;

typedef struct {
    const float* field;            /* [nz][ny][nx] */
    int32_t nx, ny, nz, brick_log2;
    const int32_t* piece_of_brick; /* [nbz*nby*nbx] */
    int32_t n_pieces, reserved;
    const uint8_t* piece_selected; /* [n_pieces], NULL = every piece */
    const float* tf;               /* [256][4] r, g, b, alpha per voxel */
    double vmin, vmax;
    double step;                   /* sample spacing, voxel units */
    double moment_bias;            /* mix amount of the bias vector (Alg. 3) */
    double overestimation;         /* weight w0 of the sample's own depth (Alg. 3) */
    double absorbance_max;         /* ABSORBANCE_MAX_VALUE (Alg. 2) */
    double bias_vector[4];
    int32_t moment_set;            /* 0: 4 power moments; 3 / 4: that many complex trigonometric moments;
                                      6 / 8: that many power moments (bias vector: orc_power_bias) */
    int32_t storage;               /* 0 FP64 moments; 1 / 2: normalised trig moments rounded to float16 / bfloat16 */
    double trig_zone;              /* zeta: angles phi = z (1 - zeta) pi leave a wrapping zone of 2 zeta pi */
} orc_grid;

typedef struct {
    const float* values;           /* [n_leaves][9][9][9]: vertex values of each leaf at its level */
    const int32_t* leaves;         /* [n_leaves][4]: origin x, y, z in finest cells, level */
    int32_t n_leaves, max_level;
    int32_t finest_cells;          /* D: the domain is [0, D]^3 in finest-cell units */
    int32_t brick_log2;            /* a leaf is 2^brick_log2 cells of its level on a side */
    const int32_t* piece_of_leaf;  /* [n_leaves] */
    int32_t n_pieces;
    int32_t adaptive_step;         /* 1: a lattice point in a leaf of level L counts only if k is a multiple
                                      of 2^(max_level - L), with absorbance sigma * step * 2^(max_level - L) */
    const uint8_t* piece_selected; /* [n_pieces], NULL = every piece */
    const float* tf;
    double vmin, vmax, step, moment_bias, overestimation, absorbance_max;
    double bias_vector[4];
    int32_t moment_set, storage;   /* as in orc_grid */
    double trig_zone;
} orc_amr;

/* Alg. 3 core: the moment-bound absorbance fraction A(z0) in [0,1] for raw
 * power moments m[0..4]; the transmittance is clamp(exp(-m[0]*A)).
 * *flags (optional) gets 1 for the one-atom, 2 for the two-atom branch. */
double orc_mboit_bound(const double m[5], double z0, double moment_bias,
                       const double bias_vector[4], double overestimation, int* flags);

/* Alg. 3 with 2n power moments, n = 2, 3 or 4 (the 4-, 6- and 8-moment
 * variants of Sec. 4.3 / Fig. 3): m = b0..b_2n raw; normalise, mix with
 * bias[0..2n-1] (b1'..b2n' of the bias measure), LDL^T of the (n+1) x (n+1)
 * Hankel matrix, q = B^-1 (1, z0, .., z0^n), the n roots of sum q_j x^j,
 * weights (overestimation at z0, indicator x_i < z0 elsewhere), the degree-n
 * polynomial interpolating them, A = p . (1, b1', .., bn').  A Hankel matrix
 * whose leading k x k block is the last positive-definite one (k <= n) means
 * a measure of k atoms, and A sums their weights.  *flags (optional): 0
 * generic, else k.  nodes (optional, n + 1 entries): z0 and the roots
 * (generic case) or the k atoms. */
double orc_power_bound(const double* m, int n, double z0, double moment_bias, const double* bias,
                       double overestimation, int* flags, double* nodes);

/* The bias measure of the 6- and 8-moment sets: moments b1..b_2n of the
 * arcsine (Chebyshev) distribution on [-1, 1], b_2k = C(2k, k) / 4^k, odd
 * moments 0.  Its Hankel matrices are positive definite at every order. */
void orc_power_bias(int n, double* bias);

/* Trigonometric moments (n = 3 or 4 complex moments, "6 / 8 trigonometric
 * moments" of Sec. 4.3 / Fig. 3): warped depth z -> angle phi = z (1 - zeta) pi,
 * moments t_j = sum a e^{i j phi}.  m = (b0, Re t1, Im t1, ..., Re tn, Im tn).
 * The bound mixes the normalised moments with the uniform measure
 * (tau'_j = (1 - beta) t_j / b0), takes the canonical representation through
 * u0 = e^{i phi0} (nodes: u0 and the roots of K(., u0), K the reproducing
 * kernel of the Toeplitz matrix; weights 1 / K(u_i, u_i)) and returns
 * w0 rho0 + the weights of the nodes at angles (in (-pi, pi]) below phi0.
 * *status (optional): 0 ok, -1 Toeplitz matrix not positive definite,
 * -2 root iteration did not converge. */
double orc_trig_bound(const double* m, int n, double phi0, double moment_bias, double overestimation,
                      int* status, double* weights_sum);

/* The canonical representation itself: nodes[2 (n+1)] (re, im; node 0 is
 * u0) and weights[n + 1].  Returns the status of orc_trig_bound. */
int orc_trig_nodes(const double* m, int n, double phi0, double moment_bias, double* nodes, double* weights);

/* Storage rounding of one normalised trigonometric moment: float64 ->
 * float32 -> float16 (storage 1) or bfloat16 (storage 2), nearest-even. */
double orc_store_round(double x, int storage);

/* Logarithmic depth warp of Alg. 2/3: [near, far] -> [-1, 1], clamped. */
double orc_log_warp(double t, double znear, double zfar);

/* Renders the listed pixels (index y*width + x) of one view.  Every output
 * pointer may be NULL.  Per pixel: moments = summed global moments [NM]
 * (NM = 1 + 2n for 2n power moments: b0..b_2n; 1 + 2n for n trigonometric
 * moments: b0, Re t1, Im t1, ...); piece_moments [K][NM]; piece_color [K][4];
 * mboit_rgba = renormalised resolve; raw_rgba = sum of T*alpha*(c,1);
 * exact_rgba = front-to-back blend of the same samples; sortlast_rgba =
 * per-piece segments sorted and blended; nsamples = owned samples.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int orc_render_grid(const orc_grid* g, const orc_view* view,
                    const int64_t* pixels, int64_t n_pixels,
                    double* moments, double* piece_moments, double* piece_color,
                    double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                    double* sortlast_rgba, int64_t* nsamples);

/* As orc_render_grid, plus nsegments[n_pixels]: segments of the sort-last
 * route (maximal runs of consecutive lattice points of one piece). */
int orc_render_grid_segments(const orc_grid* g, const orc_view* view,
                             const int64_t* pixels, int64_t n_pixels,
                             double* sortlast_rgba, int64_t* nsegments);

/* The same outputs for a brick-octree (AMR) volume: a lattice point belongs
 * to the leaf whose half-open box contains it, and takes the trilinear
 * interpolation of that leaf's vertex values at the leaf's resolution.
 * Returns -1 also for overlapping leaves. */
int orc_render_amr(const orc_amr* a, const orc_view* view,
                   const int64_t* pixels, int64_t n_pixels,
                   double* moments, double* piece_moments, double* piece_color,
                   double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                   double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments);

/* Tetrahedral mesh (Sec. 5: unstructured pieces; a piece is a set of tets).
 * Point location is exact: positions and vertices snap to the lattice of
 * multiples of 2^-quantum_log2 (nearest-even), and a snapped point q belongs
 * to the one tet containing q + (e, e^2, e^3) for an infinitesimal e > 0
 * (symbolic perturbation), so that the tets of a conforming mesh partition
 * the box exactly with no gaps or double counts on faces, edges and
 * vertices.  The value is the barycentric (linear) interpolation of the four
 * vertex values at q. */
typedef struct {
    const float* verts;            /* [n_verts][4]: x, y, z, value */
    const int32_t* tets;           /* [n_tets][4]: vertex ids, positively oriented */
    int64_t n_verts, n_tets;
    double box[3];                 /* the domain is [0, box) per axis; vertices lie in [0, box] */
    int32_t quantum_log2;
    int32_t reserved;
    const int32_t* piece_of_tet;   /* [n_tets] */
    int32_t n_pieces, reserved2;
    const uint8_t* piece_selected; /* [n_pieces], NULL = every piece */
    const float* tf;
    double vmin, vmax, step, moment_bias, overestimation, absorbance_max;
    double bias_vector[4];
    int32_t moment_set, storage;   /* as in orc_grid */
    double trig_zone;
} orc_tet;

/* The render outputs of orc_render_amr for a tetrahedral mesh.  Returns -1
 * also for a tet that is not positively oriented after snapping, a vertex
 * outside the box, or a point that two tets claim (a mesh that overlaps). */
int orc_render_tet(const orc_tet* m, const orc_view* view,
                   const int64_t* pixels, int64_t n_pixels,
                   double* moments, double* piece_moments, double* piece_color,
                   double* mboit_rgba, double* raw_rgba, double* exact_rgba,
                   double* sortlast_rgba, int64_t* nsamples, int64_t* nsegments);

/* Point location alone: for n float32 points (x, y, z), the owning tet
 * (-1: none), the number of tets that pass the test (0 or 1 for a valid
 * mesh) and the interpolated value (NaN if none).  brute_force = 1 tests
 * every tet instead of the candidates of the point's bin.  Returns 0 / -1. */
int orc_tet_locate(const orc_tet* m, const float* points, int64_t n, int32_t* tet_out, int32_t* n_pass_out,
                   double* value_out, int32_t brute_force);

/* Mixed cells (Sec. 5: the FUN3D pieces hold tetrahedra, pyramids and
 * prisms) split into tetrahedra.  cells[6 i ..]: the vertex ids of cell i,
 * types[i] = 4 (tet), 5 (pyramid: base quad in cyclic order, apex) or 6
 * (prism: bottom triangle, top triangle, vertex j + 3 above vertex j).
 * Every quad face is cut along the diagonal through its smallest vertex id,
 * so two cells sharing a face cut it alike (a conforming split): a pyramid
 * gives 2 tets, a prism 3 (the smallest id fixes which of its two
 * three-tet splits fits the three cuts).  Each tet is made positively
 * oriented on the snapped coordinates (its last two vertices swapped if
 * not).  tets_out [max_tets][4], cell_of_tet [max_tets]; *n_tets = count.
 * Returns 0, -1 on bad arguments, a flat tet or too small a buffer. */
int orc_split_cells(const float* verts, int64_t n_verts, const int32_t* cells, const int32_t* types, int64_t n_cells,
                    int32_t quantum_log2, int32_t* tets_out, int64_t* cell_of_tet, int64_t max_tets, int64_t* n_tets);

/* Stage two of the listed pixels of a grid from given global moments
 * (per pixel in the order of orc_render_grid's `moments`); writes the
 * renormalised image and / or the raw sum.  Returns -1 on bad arguments. */
int orc_render_grid_given(const orc_grid* g, const orc_view* V, const int64_t* pixels, int64_t n_pixels,
                          const double* given_moments, double* mboit_rgba, double* raw_rgba);

#ifdef __cplusplus
}
#endif
#endif
