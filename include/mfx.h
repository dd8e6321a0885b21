/*
 * mfx -- matrix-free Q_k Laplacian on hexahedral meshes, GB300 (sm_103a).
 *
 * C-ABI of libmfx.so.  The operator is the condensed stiffness operator of
 * the variable-coefficient Laplacian, i.e. the bilinear form of Eq. (1)
 * (Sec. 2.4) with a coefficient a(x):
 *
 *     a(u, v) = integral over Omega of a(x) grad u . grad v dx,
 *
 * discretised with continuous tensor-product Lagrange elements of degree k
 * on Gauss-Lobatto nodes (Sec. 3.1, Sec. 3.4), (k+1)-point Gauss quadrature
 * per direction and a trilinear (Q1) mapping of every hexahedron
 * (Sec. 3.4, mappings).  Following the matrix-free paradigm of Sec. 3.6,
 * no matrix is ever formed: the operator is applied through the weak-form
 * integrals, using the tensor-product structure of the shape functions
 * (sum factorisation, Sec. 3.6).  Constraints (homogeneous Dirichlet on the
 * box boundary, hanging nodes of locally refined meshes, Sec. 3.1 and
 * Sec. 3.3) are resolved inside the operator: on constrained DoFs the
 * operator is the identity, on free DoFs it is C^T A C where C expands free
 * values into constrained ones.
 *
 * Conventions
 *  - The library owns setup data (mesh tables, geometry) in device memory.
 *    The caller owns every vector: contiguous device arrays of n_dofs
 *    entries of the stated precision (double for MFX_F64, float for MFX_F32).
 *  - Streams are passed as opaque pointers (cudaStream_t); NULL is the
 *    legacy default stream.  vmult, diagonal and the vector calls are
 *    asynchronous on that stream and allocate nothing.
 *  - Errors never abort: every call returns an mfx_status; the message of
 *    the last error of the calling thread is returned by mfx_last_error().
 *    Asynchronous device faults surface at the next synchronising call.
 *  - DoF indices are int32 (n_dofs < 2^31); sizes are int64.
 */
#ifndef MFX_H
#define MFX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mfx_status;
enum {
  MFX_OK = 0,
  MFX_EINVAL = -1,       /* bad argument (null pointer, size, range)          */
  MFX_EUNSUPPORTED = -2, /* valid request this build does not implement        */
  MFX_ENOMEM = -3,       /* device or host allocation failed                   */
  MFX_ECUDA = -4,        /* a CUDA runtime call failed                         */
  MFX_EMESH = -5,        /* invalid mesh: holes/overlaps, not 2:1 balanced     */
  MFX_ETIMEOUT = -6,     /* a bounded device wait ran out                      */
  MFX_EBUSY = -7,        /* no capacity (admission refused)                    */
  MFX_NOT_CONVERGED = 1, /* iteration cap reached                              */
  MFX_BREAKDOWN = 2      /* NaN/Inf or non-positive curvature p.Ap <= 0        */
};

typedef enum { MFX_F64 = 0, MFX_F32 = 1 } mfx_prec;

enum { MFX_COEF_CONSTANT = 0, /* a = par[0]                                   */
       MFX_COEF_TRIG = 1,     /* a = par[0] + par[1] sin(2 pi x) cos(2 pi y) z */
       MFX_COEF_QPOINT = 2,   /* a given at every quadrature point             */
       MFX_COEF_FUNCTION = 3 }; /* a(x) from a host function at set-up         */

/* A scalar function of a physical point, evaluated on the host in FP64. */
typedef double (*mfx_point_fn)(const double x[3], void* user);
/* A map of physical points, evaluated on the host in FP64. */
typedef void (*mfx_map_fn)(const double in[3], double out[3], void* user);

enum { MFX_PRECOND_JACOBI = 0, MFX_PRECOND_CHEBYSHEV = 1 };

typedef struct mfx_mesh mfx_mesh;
typedef struct mfx_op mfx_op;
typedef void* mfx_stream; /* cudaStream_t */

/* Message of the last failed call on this thread ("" if none).  No counterpart in the paper. */
const char* mfx_last_error(void);
/* Library version string (static storage).  No counterpart in the paper. */
const char* mfx_version(void);

/*
 * Structured box mesh of nx*ny*nz hexahedra (Sec. 3.1).
 * vertices: host, (nx+1)(ny+1)(nz+1) x 3 doubles, lexicographic with x
 * fastest; NULL means the unit cube lattice (i/nx, j/ny, l/nz).  Copied.
 * Cells are lexicographic (x fastest); cell vertex v = a + 2b + 4c is the
 * corner (a, b, c).  Every DoF on the box boundary is Dirichlet (u = 0).
 * Errors: MFX_EINVAL for non-positive sizes or a null out pointer.
 */
mfx_status mfx_mesh_create_structured(mfx_mesh** out, int32_t nx, int32_t ny, int32_t nz,
                                      const double* vertices);

/*
 * Octree mesh (local refinement with hanging nodes, Sec. 3.1, Fig. 2).
 * coarse_vertices: as for the structured mesh (NULL = unit cube).
 * leaves: host, n_leaves x 4 int32 (level, i, j, l), the leaf covering
 * [i, i+1] x [j, j+1] x [l, l+1] in units of 1/(n 2^level) coarse cells;
 * levels 0..8.  Leaves must tile the coarse box exactly and be 2:1
 * balanced across faces and edges, else MFX_EMESH.  Cells are ordered by
 * (coarse cell lexicographic, Morton order within the tree, x bit lowest);
 * leaf vertices are the trilinear map of the coarse cell at the leaf's
 * reference corners.  DoFs are numbered on first encounter (cells in order,
 * local nodes lexicographic); coincident nodes share one DoF.  Hanging
 * nodes are constrained to the coarse face (edge) nodes with Lagrange
 * weights; Dirichlet takes precedence; Dirichlet masters and zero weights
 * are dropped; masters are sorted by DoF.  Input arrays are copied.
 */
mfx_status mfx_mesh_create_octree(mfx_mesh** out, int32_t nx, int32_t ny, int32_t nz,
                                  const double* coarse_vertices, const int32_t* leaves,
                                  int64_t n_leaves);
void mfx_mesh_destroy(mfx_mesh* mesh);

/*
 * Boundary conditions: bit 2d of `faces` (d = 0 x, 1 y, 2 z) makes the box face at coordinate 0
 * a homogeneous Dirichlet face (u = 0), bit 2d + 1 the face at the far end; the other faces are
 * natural (Neumann, zero flux) boundaries of the weak form.  Default 0x3F (all six faces).  The
 * constrained set (and with it the tables, the identity rows of the operator and the diagonal)
 * follows the mask; operators built earlier keep theirs.  A DoF on several faces is Dirichlet if
 * any of them is.  With no Dirichlet face the operator is singular (constants are in its kernel).
 * The Dirichlet constraints are those of Sec. 3.3 (constrained DoFs with no masters), the natural
 * faces the boundary term that the weak form of Eq. 1 (Sec. 2.4) drops.
 * Errors: MFX_EINVAL (null mesh, faces > 0x3F).
 */
enum { MFX_FACE_X0 = 1, MFX_FACE_X1 = 2, MFX_FACE_Y0 = 4, MFX_FACE_Y1 = 8, MFX_FACE_Z0 = 16,
       MFX_FACE_Z1 = 32, MFX_FACES_ALL = 63 };
mfx_status mfx_mesh_set_dirichlet(mfx_mesh* mesh, uint32_t faces);
mfx_status mfx_mesh_get_dirichlet(const mfx_mesh* mesh, uint32_t* faces);

/*
 * Move the mesh: every vertex v of the vertex lattice (structured) or of the
 * coarse lattice (octree) becomes phi(v), evaluated on the host in FP64
 * (the geometry is given by the moved vertices and the trilinear map of each
 * cell, Sec. 3.4).  Octree leaf vertices follow from the moved coarse cells'
 * trilinear maps, so leaves stay conforming.  Operators built earlier keep
 * their geometry.  Errors: MFX_EINVAL (null mesh or map).
 */
mfx_status mfx_mesh_transform(mfx_mesh* mesh, mfx_map_fn phi, void* user);

/*
 * Host-only (no GPU needed): sizes of the DoF and constraint tables of the
 * mesh at degree k (numbering and constraint rules as described above: the
 * DoF enumeration of Sec. 3.1 / Sec. 3.4 and the constraints of Sec. 3.3).
 * Any output pointer may be NULL.
 * Errors: MFX_EINVAL, MFX_EUNSUPPORTED (k out of 1..8), MFX_EMESH.
 */
mfx_status mfx_mesh_table_sizes(const mfx_mesh* mesh, int32_t degree, int64_t* n_cells, int64_t* n_dofs,
                                int64_t* n_constrained, int64_t* n_masters);

/*
 * Host-only: the tables themselves (Sec. 3.1, Sec. 3.3), laid out as for mfx_get_tables below
 * (caller-allocated host arrays of the sizes above; NULL skips a table).
 * Errors: MFX_EINVAL, MFX_EUNSUPPORTED (k out of 1..8), MFX_EMESH.
 */
mfx_status mfx_mesh_tables(const mfx_mesh* mesh, int32_t degree, int32_t* cell_dofs, int32_t* constrained,
                           int64_t* cptr, int32_t* cmaster, double* cweight);

/*
 * Host-only: the hanging-node constraints of an octree mesh at degree k in the
 * tensor-product form the octree vmult applies for k >= 3 (Sec. 3.3, Fig. 2:
 * the values on a refined cell's face or edge that lies on a coarser
 * neighbour's face or edge are that neighbour's polynomial there).  Per cell:
 *   hface[c]  bit f set if face f (f = 2 d + side, d = 0,1,2 for x,y,z) lies
 *             on a coarser neighbour's face; bits 6 + 2 f and 7 + 2 f give
 *             the half (0 lower, 1 upper) of the coarse face it covers along
 *             its first and second tangential direction (u, v: the lower and
 *             the higher of the two other axes);
 *   hedge[c]  bit e set if edge e (e = 4 d + 2 side_v + side_u, along axis d)
 *             lies on a coarser cell's edge and on no hanging face of the
 *             cell; bit 12 + e gives the half of the coarse edge it covers;
 *   hoff[c]   start in hdofs of the cell's coarse DoFs: for each hanging
 *             face in f order the (k+1)^2 DoFs of the coarse face (u fastest),
 *             then for each hanging edge in e order the k+1 DoFs of the coarse
 *             edge; a coarse DoF that is itself constrained is stored as -1.
 * A constrained node of the cell on a hanging face (the first in f order)
 * takes the value  sum_mu,mv l_mu((cu + x_bu)/2) l_mv((cv + x_bv)/2) u_mu,mv
 * of the coarse face values, with x_b its GLL coordinates on the face and
 * l the GLL Lagrange basis; one on a hanging edge only the 1D analogue.
 * Caller-allocated host arrays: hface, hedge, hoff n_cells entries, hdofs
 * *n_hdofs entries (call once with hdofs = NULL to get the count); NULL skips
 * an array.  Structured meshes: all zero, *n_hdofs = 0.
 * Errors: MFX_EINVAL, MFX_EUNSUPPORTED (k out of 1..8), MFX_EMESH.
 */
mfx_status mfx_mesh_hanging_tables(const mfx_mesh* mesh, int32_t degree, uint32_t* hface, uint32_t* hedge,
                                   int64_t* hoff, int32_t* hdofs, int64_t* n_hdofs);

typedef struct {
  int32_t degree;        /* k, 1..8                                               */
  int32_t n_q_1d;        /* quadrature points per direction; 0 or k+1 (only k+1)  */
  int32_t coef_kind;     /* MFX_COEF_*                                            */
  int32_t precisions;    /* bit 0: FP64 data, bit 1: FP32 data; 0 means both      */
  double coef_par[2];    /* parameters of the coefficient                         */
  const double* coef_qpoint; /* MFX_COEF_QPOINT: device, n_cells x n_q^3 doubles,
                                q = q1 + n_q (q2 + n_q q3); read during create  */
  int32_t cells_per_block;   /* 0 = autotuned default                             */
  int32_t discretization;    /* MFX_CONTINUOUS (0) or MFX_SIPG (1)                 */
  mfx_point_fn coef_fn;      /* MFX_COEF_FUNCTION: a(x), called once per quadrature
                                point during create (on the calling thread)      */
  void* coef_user;
  double dg_penalty;         /* MFX_SIPG: eta of the penalty (0 means 1)            */
  int32_t structured_kernel; /* FP32 vmult kernel of a structured continuous
                                operator at k = 1..4: MFX_KERNEL_* (0 = autotuned)  */
} mfx_op_desc;

/*
 * Kernels of the FP32 vmult on structured meshes (the cell loop of Sec. 3.6; the choice does not
 * change the result beyond rounding).  TEN_PHASE: collocation derivative after the interpolation
 * to the Gauss points, ten synchronised sweeps per batch of cells.  FIVE_PHASE: values and
 * derivatives of the nodal basis at the Gauss points taken from the same line in each sweep
 * (sixteen 1D contractions per line in five synchronised sweeps), metric read where it is used;
 * FIVE_PHASE_STAGED: the same with each batch's metric copied into shared memory first.
 * Degrees above 4 always use their own kernels.  No counterpart in the paper.
 */
enum { MFX_KERNEL_AUTO = 0, MFX_KERNEL_TEN_PHASE = 1, MFX_KERNEL_FIVE_PHASE = 2, MFX_KERNEL_FIVE_PHASE_STAGED = 3 };

/*
 * MFX_SIPG: the symmetric interior penalty DG Laplacian of the paper's multigrid benchmark
 * (Sec. 6.1) on a structured mesh of uniform, axis-aligned cells (the lattice must be
 * x_i = x_0 + i h per direction, else MFX_EUNSUPPORTED) with a constant coefficient a = par[0]:
 * discontinuous Q_k on Gauss-Lobatto nodes, DoFs cell-major (n_cells x (k+1)^3, cell c's node
 * i1 + n (i2 + n i3) at c n^3 + ...), interior faces -{d_n u}[v] - [u]{d_n v} + sigma [u][v] with
 * sigma = eta (k+1)^2 / h, homogeneous Dirichlet data imposed weakly on the mesh's Dirichlet faces
 * (sigma = 2 eta (k+1)^2 / h there), the other faces natural.  There are no constrained DoFs.
 * vmult, diagonal, dot, Chebyshev, solve, batches, quadrature points and right-hand sides
 * (mfx_rhs, mfx_rhs_function: b_i = integral of f phi_i over phi_i's cell) work as for the
 * continuous operator; mfx_get_tables returns the identity cell-to-DoF map and no constraints.
 */
enum { MFX_CONTINUOUS = 0, MFX_SIPG = 1 };

/*
 * Build the operator: DoF tables and constraints on the host, then the
 * per-quadrature-point geometry on the device in FP64 (Jacobian of the Q1
 * map, det J, J^-1, coefficient at the physical point) merged into the
 * symmetric 3x3 metric a |det J| w_q J^-1 J^-T (plus an FP32 copy), and the
 * diagonal of the operator.  This is the set-up of the matrix-free operator of
 * Sec. 3.6 (geometry precomputed at the quadrature points) for the mesh,
 * element, mapping and quadrature of Sec. 3.4.  Synchronises the stream.
 * Errors: MFX_EINVAL, MFX_EUNSUPPORTED (k > 8, n_q != k+1), MFX_EMESH,
 * MFX_ENOMEM, MFX_ECUDA.
 */
mfx_status mfx_operator_create(mfx_op** out, const mfx_mesh* mesh, const mfx_op_desc* desc,
                               mfx_stream stream);
/* Frees the operator after waiting for all work on the device (safe whatever is still queued).
 * No counterpart in the paper. */
void mfx_operator_destroy(mfx_op* op);
/*
 * Frees the operator without waiting for the device: its memory (and its solver workspace) is
 * released in stream order on `stream`.  The caller guarantees that every piece of work that uses
 * the operator is complete or ordered before `stream`'s current position (for example: a batch slot
 * that mfx_batch_poll reported done).  No counterpart in the paper: it exists so that a serving
 * loop can drop finished problems without a device-wide synchronisation.
 * Errors: MFX_EINVAL (null operator).  The handle is invalid afterwards.
 */
mfx_status mfx_operator_release(mfx_op* op, mfx_stream stream);
/*
 * Allocates the operator's solver workspace now (nine vectors per stored precision, stream-ordered
 * device memory) instead of at the first mfx_solve / mfx_batch_add, so that a set-up thread can pay
 * for it.  No counterpart in the paper.  Synchronises the workspace's own stream.
 * Errors: MFX_EINVAL (null operator, no FP64 data), MFX_ENOMEM, MFX_ECUDA.
 */
mfx_status mfx_solver_prepare(mfx_op* op);

typedef struct {
  int64_t n_dofs, n_cells, n_constrained, n_masters, n_hanging;
  int64_t bytes_device; /* device memory owned by the operator */
  int32_t degree, n_q_1d, structured, cells_per_block;
  int32_t discretization;  /* MFX_CONTINUOUS or MFX_SIPG */
  int32_t structured_kernel; /* MFX_KERNEL_* of the FP32 structured vmult (0 where none applies) */
  int32_t box_metric;  /* 1: an octree operator whose cells are all axis-aligned boxes with a constant
                          coefficient, whose FP32 kernels take the metric as one diagonal per cell */
  int32_t reserved;
} mfx_op_info;

/*
 * Sizes and layout of an operator: the DoF count of the Q_k space on the mesh
 * (Sec. 3.1 and Sec. 3.4), the cells, the constrained DoFs and constraint
 * entries of the hanging-node and Dirichlet constraints (Sec. 3.3), the
 * device bytes, and the chosen batch size and FP32 kernel (these three
 * have no counterpart in the paper), and whether the FP32 metric is stored
 * per box cell (the specialised mapping of cells that are boxes with axes
 * parallel to the coordinate axes, Sec. 2).  Errors: MFX_EINVAL (null argument).
 */
mfx_status mfx_operator_info(const mfx_op* op, mfx_op_info* info);

/*
 * Host copies of the integer and constraint tables (for bit-exact checks):
 * the enumeration of the DoFs of each cell (Sec. 3.1, Sec. 3.4) and the
 * constraints of hanging nodes and Dirichlet boundaries (Sec. 3.3, Fig. 2:
 * each constrained DoF a weighted sum of masters, Dirichlet DoFs none).
 * cell_dofs: n_cells x (k+1)^3 (local i1 + n (i2 + n i3)); constrained:
 * n_constrained sorted DoFs; cptr: n_constrained + 1; cmaster, cweight:
 * n_masters.  Any pointer may be NULL to skip that table.  Caller-owned host
 * arrays of those sizes (mfx_operator_info gives them).  Synchronous.
 * Errors: MFX_EINVAL (null operator).
 */
mfx_status mfx_get_tables(const mfx_op* op, int32_t* cell_dofs, int32_t* constrained, int64_t* cptr,
                          int32_t* cmaster, double* cweight);

/*
 * dst = K src (Sec. 3.6): per cell, gather with constraint resolution,
 * interpolate to the Gauss points and take reference gradients by 1D
 * contractions, apply the stored metric, integrate back with the
 * transposed contractions, scatter-add; constrained rows copy src.
 * src, dst: device, n_dofs entries of the precision, must not alias; on
 * structured meshes the FP32 kernels move tile rows with the copy engine and
 * need src and dst 16-byte aligned (as cudaMalloc and torch give them).
 * SIPG operators take vectors of any alignment; in FP32 at degrees 1..5
 * their fastest kernel stages src with 16-byte copies and runs when src is
 * 16-byte aligned (otherwise the line kernel runs, same result to rounding).
 * Errors: MFX_EINVAL (null, precision not built, or an FP32 vector on a
 * structured mesh not 16-byte aligned), MFX_ECUDA (launch).
 */
mfx_status mfx_vmult(const mfx_op* op, mfx_prec prec, const void* src, void* dst, mfx_stream stream);
/*
 * dst[i] = K src[i] for `count` vectors in HOST memory (pinned for full speed; pageable works,
 * with staged copies).  The vectors go through a three-stage pipeline on the library's own streams:
 * the upload of vector i + 1, the vmult of vector i and the download of vector i - 1 overlap, with
 * double-buffered device staging (allocated stream-ordered per call).  The call waits for the
 * work already queued on `stream` before it starts and returns once every result is in host
 * memory.  src[i], dst[i]: n_dofs entries of the precision; no dst[i] may alias a src[j].
 * No counterpart in the paper: this is the host-buffer path of the operator.
 * Errors: MFX_EINVAL (null, count < 0, precision not built), MFX_ENOMEM, MFX_ECUDA.
 */
mfx_status mfx_vmult_host(const mfx_op* op, mfx_prec prec, int32_t count, const void* const* src,
                          void* const* dst, mfx_stream stream);

/*
 * Synchronise the stream and report device-side failures of this operator's
 * kernels: MFX_ETIMEOUT if a bounded wait inside a kernel ran out (the word
 * is then cleared), MFX_ECUDA for a CUDA error, else MFX_OK.  No counterpart
 * in the paper (failure detection of this library's kernels).
 */
mfx_status mfx_device_check(const mfx_op* op, mfx_stream stream);

/*
 * Self-test of the failure detection above, without a fault: launches one
 * CTA that waits on a shared-memory mbarrier at which nothing ever arrives,
 * through the same bounded wait (about 2^31 SM clocks, about one second)
 * that the TMA kernels use.  The wait runs out, the kernel sets the
 * operator's error word and returns; the next mfx_device_check on the
 * stream reports MFX_ETIMEOUT (and clears the word), and the operator stays
 * usable.  Asynchronous on stream.  No counterpart in the paper.
 * Errors: MFX_EINVAL (null operator), MFX_ECUDA.
 */
mfx_status mfx_selftest_bounded_wait(const mfx_op* op, mfx_stream stream);

/*
 * Checked mode (in place of a memory checker; no counterpart in the paper; the
 * tables are those of Sec. 3.1 and Sec. 3.3).  Index tables as the
 * per-cell kernels read them, all device arrays:
 *   cell_dofs  n_cells x nodes_1d^3 codes: a DoF in [0, n_dofs), or -1 - r
 *              for constraint row r in [0, n_rows);
 *   cptr       n_rows + 1 row pointers into cmaster (0 first, non-
 *              decreasing, n_masters last); NULL when n_rows = 0;
 *   cmaster    n_masters master DoFs in [0, n_dofs);
 *   hface, hedge, hoff, hdofs  the tensor-product hanging tables of
 *              mfx_mesh_hanging_tables (n_cells words and offsets, n_hdofs
 *              codes in [-1, n_dofs)); hface = NULL skips them;
 *   cell_list[l]  n_list[l] cell indices in [0, n_cells) (NULL when 0).
 * mfx_validate_tables checks every entry on the device, reading each array
 * only below its stated size, and returns MFX_EMESH with *n_bad = the number
 * of entries out of range or inconsistent (a hanging word with undefined
 * bits, or whose slots do not end where the next cell's start), else MFX_OK
 * and *n_bad = 0 (n_bad may be NULL).  Synchronises the stream.
 * mfx_operator_validate applies it to an operator's own device tables
 * (octree meshes, and structured meshes whose FP32 vmult uses a lattice
 * table; nothing to check otherwise).  With the environment variable
 * MFX_CHECKED set (not "0"), mfx_operator_create runs it before returning
 * and fails with its status.
 * Errors: MFX_EINVAL (null descriptor or operator, negative size, a table
 * with entries but a null pointer), MFX_EMESH, MFX_ECUDA.
 */
typedef struct {
  int64_t n_cells;
  int32_t nodes_1d;      /* k + 1 */
  int32_t reserved;
  int64_t n_dofs, n_rows, n_masters, n_hdofs;
  const int32_t* cell_dofs;
  const int64_t* cptr;
  const int32_t* cmaster;
  const uint32_t* hface;
  const uint32_t* hedge;
  const int64_t* hoff;
  const int32_t* hdofs;
  const int32_t* cell_list[2];
  int64_t n_list[2];
} mfx_index_tables;
mfx_status mfx_validate_tables(const mfx_index_tables* tables, int64_t* n_bad, mfx_stream stream);
mfx_status mfx_operator_validate(const mfx_op* op, int64_t* n_bad, mfx_stream stream);

/*
 * diag = diagonal of K (1 on constrained rows), device, n_dofs entries of the
 * precision: the Jacobi preconditioner of the CG solve and the diagonal of
 * the Chebyshev smoother (Sec. 3.5, Sec. 6.1), computed in FP64 when the
 * operator is created.  Asynchronous on stream.
 * Errors: MFX_EINVAL (null, precision not built).
 */
mfx_status mfx_diagonal(const mfx_op* op, mfx_prec prec, void* diag, mfx_stream stream);

/*
 * Physical quadrature points (the mapping of Sec. 3.4 applied to the tensor
 * Gauss points of each cell), device, n_cells x n_q^3 x 3 doubles, q = q1 +
 * n_q (q2 + n_q q3), caller-allocated.  Asynchronous on stream.
 * Errors: MFX_EINVAL (null argument).
 */
mfx_status mfx_quadrature_points(const mfx_op* op, double* xq, mfx_stream stream);

/*
 * Right-hand side of the step-4 cell loop (Sec. 2.4): b_i = sum_q phi_i f_q
 * |det J_q| w_q assembled and condensed (C^T b, 0 on constrained DoFs).
 * fq: device, n_cells x n_q^3 doubles; b: device, n_dofs doubles.
 */
mfx_status mfx_rhs(const mfx_op* op, const double* fq, double* b, mfx_stream stream);
/*
 * The same load vector for f given as a host function: f is evaluated on the
 * host at the physical quadrature points (as returned by
 * mfx_quadrature_points), then integrated as mfx_rhs does.  Synchronises the
 * stream.  Errors: MFX_EINVAL, MFX_ENOMEM, MFX_ECUDA.
 */
mfx_status mfx_rhs_function(const mfx_op* op, mfx_point_fn f, void* user, double* b, mfx_stream stream);

/*
 * Fill constrained entries of x (device, FP64, n_dofs) from the free ones:
 * hanging DoFs get their weighted masters (the constraint rows of Sec. 3.3),
 * Dirichlet DoFs 0.  Asynchronous on stream.  Errors: MFX_EINVAL (null).
 */
mfx_status mfx_distribute(const mfx_op* op, double* x, mfx_stream stream);

/* ---------------------------------------------------------------- vectors */

/*
 * result[0] = sum_i a_i b_i, accumulated in FP64 in a fixed order (device
 * scalar): the inner products of the CG solve with the multigrid or
 * Chebyshev preconditioner and of the double-precision correction (Sec.
 * 6.1).  a, b: device vectors of n entries of the precision.  The
 * reduction partials live in scratch memory owned by the operator, so
 * calls on one operator must not overlap on the GPU.
 * Errors: MFX_EINVAL (null, n < 0).
 */
mfx_status mfx_dot(const mfx_op* op, mfx_prec prec, int64_t n, const void* a, const void* b,
                   double* result, mfx_stream stream);

/*
 * Allocation-free variant of mfx_dot (the paper has no counterpart).  It serves
 * callers that cannot call cudaMalloc: a plug-in whose host application owns all
 * device memory, code that runs inside another runtime's memory pool, or a loop
 * that must not block on the allocator.  Same result as mfx_dot, without an
 * operator: the reduction partials live in a fixed array of about 8 KB compiled
 * into the library (kept on every GPU that loads it until exit).
 * a, b: device vectors of n entries of the precision; result: device FP64 scalar.
 * n above MFX_NOALLOC_MAX_N is rejected with MFX_EINVAL.  The first call on a device
 * looks up the array's address (cudaGetSymbolAddress).  Calls share the array: calls
 * that overlap on the GPU race and give wrong results.
 */
#define MFX_NOALLOC_MAX_N 2147483647LL
mfx_status mfx_dot_noalloc(mfx_prec prec, int64_t n, const void* a, const void* b, double* result,
                           mfx_stream stream);

/*
 * Chebyshev-Jacobi preconditioner (smoother named in Sec. 3.5 and Sec. 6.1):
 * z = p(D^-1 K) D^-1 r with 1 - lambda p(lambda) = T_m(s(lambda)) / T_m(s(0)),
 * s(lambda) = (hi + lo - 2 lambda) / (hi - lo), m = degree >= 1, computed by
 * m steps of the Chebyshev iteration from z = 0 (m - 1 operator products).
 * r, z: device vectors of the precision (must not alias).  Uses operator
 * workspace; calls on one operator must not overlap.
 */
mfx_status mfx_chebyshev(const mfx_op* op, mfx_prec prec, const void* r, void* z, int32_t degree,
                         double lo, double hi, mfx_stream stream);

/* ------------------------------------------------------------------ solve */

typedef struct {
  double tol;            /* relative residual ||b - Kx|| <= tol ||b|| (default 1e-10) */
  int32_t max_it;        /* iteration cap (outer cap for mixed), default 100000     */
  int32_t precond;       /* MFX_PRECOND_JACOBI or MFX_PRECOND_CHEBYSHEV              */
  int32_t cheb_degree;   /* Chebyshev degree (default 5)                             */
  int32_t mixed;         /* 0: FP64 PCG; 1: FP32 PCG inside FP64 defect correction   */
  double inner_tol;      /* inner relative tolerance for mixed (default 1e-4)        */
  int32_t check_every;   /* convergence checked on the host every m iterations (0=auto) */
  int32_t lanczos_steps; /* CG steps for the eigenvalue estimate (default 15)        */
  double cheb_lo, cheb_hi; /* Chebyshev interval of D^-1 K; 0 = estimate            */
  const double* lanczos_start; /* device start vector for the estimate; NULL = b     */
  int32_t inner_max_it;  /* inner cap for mixed (default 10000)                      */
  int32_t reserved;
} mfx_solve_params;

typedef struct {
  int32_t status;        /* MFX_OK, MFX_NOT_CONVERGED or MFX_BREAKDOWN             */
  int32_t iterations;    /* PCG iterations (FP64 solve) or outer corrections (mixed) */
  int32_t inner_iterations; /* total FP32 PCG iterations (mixed)                    */
  int32_t reserved;
  double rel_residual;   /* final ||b - Kx|| / ||b|| in FP64                        */
  double lambda_max;     /* eigenvalue estimate used for Chebyshev (0 if none)     */
  double cheb_lo, cheb_hi;
  double seconds;        /* wall time of the call (mfx_solve, mfx_mg_solve)         */
} mfx_solve_stats;

/* Fill params with the defaults listed above (this library's choices; the paper states none). */
void mfx_solve_params_default(mfx_solve_params* params);

/*
 * Solve K x = b (x0 = 0).  FP64 PCG with Jacobi or Chebyshev-Jacobi, or
 * (mixed = 1) FP64 defect correction around an FP32 PCG (the single-
 * precision solver with a double-precision correction of Sec. 6.1).  The
 * Krylov loop runs on the device; the host reads a status word every
 * check_every iterations.  b, x: device FP64.  Synchronises the stream.
 */
mfx_status mfx_solve(const mfx_op* op, const double* b, double* x, const mfx_solve_params* params,
                     mfx_solve_stats* stats, mfx_stream stream);

/* ---------------------------------------------------------------- batches */

/*
 * A batch advances many independent solves together (workload: many small
 * problems of uneven size, or a stream of requests).  Each slot holds one
 * operator and runs the mixed-precision solve of mfx_solve (mixed = 1:
 * FP64 residual and update, FP32 PCG inner solve) or the FP64 PCG
 * (mixed = 0).  One call to mfx_batch_step is one scheduler tick: FP64
 * residuals of the slots between inner solves, then ONE graph launch whose
 * child graphs advance every slot in an inner solve by `chunk` iterations
 * (the slots' kernels overlap on the GPU), then bookkeeping.  Problems may be
 * added and released between ticks.  x0 = 0; stopping rules as mfx_solve.
 * An operator may be in one active slot at a time (else MFX_EBUSY).
 * No counterpart in the paper: batching is this library's; each slot's solve
 * is the mixed-precision or FP64 solve of mfx_solve (Sec. 6.1).
 * Errors of every mfx_batch_* call: MFX_EINVAL (null, bad slot or size),
 * MFX_EBUSY, MFX_ENOMEM, MFX_ECUDA.
 */
typedef struct mfx_batch mfx_batch;
mfx_status mfx_batch_create(mfx_batch** out, int32_t max_slots, int32_t chunk);
void mfx_batch_destroy(mfx_batch* batch);
/* Add a solve of K x = b (b, x device FP64, caller-owned until released); returns its slot.
 * Queues ||b||^2 and x = 0 on the slot's stream and captures its iteration graph; it does not wait
 * for the GPU (the solver workspace is allocated here unless mfx_solver_prepare made it). */
mfx_status mfx_batch_add(mfx_batch* batch, const mfx_op* op, const double* b, double* x,
                         const mfx_solve_params* params, int32_t* slot);
/* One scheduler tick (synchronising); n_active = slots still running. */
mfx_status mfx_batch_step(mfx_batch* batch, int32_t* n_active);
/*
 * Independent stepping (for mixes of very different problems): every slot
 * whose previous work has finished takes its next step at once (residual,
 * stopping decision, inner start, next chunk of iterations), each slot on
 * its own stream; the call does not wait for the GPU.  Call it repeatedly;
 * n_active = slots still running.  Do not mix with mfx_batch_step on the
 * same slots while work is in flight.
 */
mfx_status mfx_batch_advance(mfx_batch* batch, int32_t* n_active);
/*
 * Every active slot's whole solve, from x = 0, in ONE graph launch.  Each slot is a graph WHILE loop
 * whose condition a kernel sets on the device: for mixed = 1 the outer defect-correction loop (FP64
 * residual and stopping test, FP32 PCG inner solve, FP64 correction) with the inner PCG loop nested in
 * it, for mixed = 0 the PCG loop; so the device decides when each problem stops, and the slots run
 * concurrently.  Every loop also ends after a capped number of passes (max_it outer passes; inner_max_it
 * or max_it iterations in chunks), so the launch always ends.  Synchronises; every slot run is done
 * afterwards (mfx_batch_poll gives its statistics).  n_done (may be NULL): the slots run.  Built and
 * launched per call (nothing persists between calls).  No counterpart in the paper.
 */
mfx_status mfx_batch_run(mfx_batch* batch, int32_t* n_done);
/* done = 1 once the slot's solve has finished; stats as mfx_solve (iterations: outer for mixed). */
mfx_status mfx_batch_poll(mfx_batch* batch, int32_t slot, int32_t* done, mfx_solve_stats* stats);
/* Free a slot (its operator and vectors can then be reused or destroyed). */
mfx_status mfx_batch_release(mfx_batch* batch, int32_t slot);

/* ---------------------------------------------------------------- multigrid */

/*
 * Geometric multigrid (the paper's large-scale solver: conjugate gradients
 * preconditioned by a multigrid V-cycle with Chebyshev smoothing and
 * matrix-free level transfers, Sec. 3.5 and Sec. 6.1), for structured meshes.
 * Levels: the given mesh and coarser ones with half the cells per direction,
 * while all three counts are even (or up to max_levels; a 2:1:1 box of
 * 2^(l+1) x 2^l x 2^l cells ends on the paper's 2 x 1 x 1 coarse mesh); a
 * coarser level's vertices are every other vertex of the finer lattice; every
 * level has the operator of `desc` (same degree, coefficient kind, Dirichlet
 * faces).  Prolongation interpolates the coarse Q_k function at the fine
 * nodes (sum-factorised per coarse cell), restriction is its transpose.  The
 * V-cycle for K_l x = b: x = S(b); x += P V_{l-1}(P^T (b - K x));
 * x += S(b - K x), with S the Chebyshev(degree) polynomial in D^-1 K on
 * [hi / range, hi], hi = 1.2 x the Lanczos estimate of each level; the
 * coarsest level is solved exactly (dense inverse of its free block).  The
 * cycle is a symmetric linear operator (identity on constrained rows).
 * desc->discretization = MFX_SIPG: the hierarchy of the paper's DG benchmark
 * (Sec. 6.1): the SIPG operator of the mesh on top, then the continuous
 * operators of the same degree on the same mesh and the coarsened ones; the
 * top transfer is the injection of the continuous space (the continuous
 * value at each DG node, Dirichlet nodes 0) and its transpose.  n_levels
 * counts the SIPG level.
 * Errors: MFX_EINVAL, MFX_EUNSUPPORTED (octree mesh, MFX_COEF_QPOINT, a
 * coarsest level above 8192 free DoFs, SIPG on a non-uniform lattice or with
 * a variable coefficient), MFX_ENOMEM, MFX_ECUDA.
 */
typedef struct mfx_mg mfx_mg;
typedef struct {
  int32_t max_levels;       /* 0: as many as the halving rule allows                 */
  int32_t smoother_degree;  /* Chebyshev degree of each smoothing step (default 6)   */
  double smoothing_range;   /* lo = hi / range (default 20)                         */
  int32_t lanczos_steps;    /* steps of the eigenvalue estimate per level (15)       */
  int32_t reserved;
} mfx_mg_params;
/* Defaults of the hierarchy: Chebyshev degree 6 on every level as in Sec. 6.1; range 20 and 15
 * Lanczos steps are this library's readings (the paper states neither). */
void mfx_mg_params_default(mfx_mg_params* params);
/* Builds the hierarchy above (Sec. 3.5, Sec. 6.1); synchronises the stream. */
mfx_status mfx_mg_create(mfx_mg** out, const mfx_mesh* mesh, const mfx_op_desc* desc, const mfx_mg_params* params,
                         mfx_stream stream);
/* Frees the hierarchy and its level operators after waiting for the device (no counterpart in the paper). */
void mfx_mg_destroy(mfx_mg* mg);
/* Number of levels and free DoFs of the coarsest level (the coarse solve of Sec. 3.5).
 * Errors: MFX_EINVAL (null argument). */
mfx_status mfx_mg_info(const mfx_mg* mg, int32_t* n_levels, int32_t* coarse_free_dofs);
/* The operator of a level (0 = coarsest, n_levels - 1 = the given mesh) of the level hierarchy of Sec. 3.5;
 * owned by the hierarchy; NULL for a level out of range. */
const mfx_op* mfx_mg_operator(const mfx_mg* mg, int32_t level);
/* Chebyshev interval of a level's smoother (levels >= 1; the Chebyshev smoothing of Sec. 3.5 and Sec. 6.1);
 * set replaces the Lanczos-based one.  Errors: MFX_EINVAL (null, level out of range, lo >= hi). */
mfx_status mfx_mg_get_bounds(const mfx_mg* mg, int32_t level, double* lo, double* hi);
mfx_status mfx_mg_set_bounds(mfx_mg* mg, int32_t level, double lo, double hi);
/* z = V(r) on the finest level, the V-cycle of Sec. 3.5 and Sec. 6.1 (device vectors of its precision,
 * not aliased); asynchronous.  Errors: MFX_EINVAL (null, precision not built), MFX_ECUDA. */
mfx_status mfx_mg_vcycle(mfx_mg* mg, mfx_prec prec, const void* r, void* z, mfx_stream stream);
/* mfx_solve on the finest operator with the V-cycle as preconditioner, the solver of Sec. 6.1
 * (params.precond is ignored; mixed = 1: FP32 PCG with the FP32 V-cycle inside FP64 defect correction,
 * the single-precision cycle with a double-precision correction of Sec. 6.1). */
mfx_status mfx_mg_solve(mfx_mg* mg, const double* b, double* x, const mfx_solve_params* params,
                        mfx_solve_stats* stats, mfx_stream stream);

/* ------------------------------------------------------------- partitions */

/*
 * Partitioned operator (the distributed path of Sec. 2.6 and Sec. 3.7: one part of the mesh per GPU,
 * each adding its neighbours' contributions on the DoFs they share).  A structured box of nx x ny x nz
 * cells is split into n_parts slabs of whole cells along z (part p gets nz / n_parts cells, one more
 * for the first nz % n_parts parts).  Part p's lattice is a contiguous slice of the global DoF vector,
 * entries dof0 .. dof0 + n_dofs - 1; its first `plane` entries are shared with part p - 1 (has_lo) and
 * its last `plane` entries with part p + 1 (has_hi).  Build the part's operator from
 * mfx_mesh_create_structured(nx, ny, nz_part, global_vertices + 3 * vertex0) with Dirichlet faces
 * `dirichlet` (the global mask without the interface faces, which are natural on the part).  On a
 * shared DoF each part's vmult then gives its own cells' contribution; adding the neighbour's
 * (mfx_halo_accumulate) gives the global operator's row.  A part owns its lattice without its upper
 * shared plane (n_owned entries, a prefix of the slice), so sums over the owned entries of all parts
 * count every DoF once.  Host-only, no GPU needed.
 * Errors: MFX_EINVAL (null info, empty box, n_parts outside 1..nz, part outside 0..n_parts - 1, mask
 * above 0x3F), MFX_EUNSUPPORTED (degree outside 1..8).
 */
typedef struct {
  int32_t cz0, nz;          /* the part's cells along z: cz0 .. cz0 + nz - 1                  */
  uint32_t dirichlet;       /* Dirichlet faces of the part's box                              */
  int32_t has_lo, has_hi;   /* a neighbour below / above                                      */
  int32_t reserved;
  int64_t dof0, n_dofs;     /* the part's lattice in the global DoF vector                   */
  int64_t n_owned;          /* owned DoFs: the first n_owned entries of the part's lattice    */
  int64_t plane;            /* DoFs of one shared lattice plane ((k nx + 1)(k ny + 1))       */
  int64_t vertex0;          /* index of the part's first vertex in the global vertex lattice  */
} mfx_part_info;
mfx_status mfx_partition_box(int32_t nx, int32_t ny, int32_t nz, int32_t degree, uint32_t dirichlet, int32_t n_parts,
                             int32_t part, mfx_part_info* info);

/*
 * The exchange step of the partitioned vmult: y's shared plane on `side` (0: the first `plane` entries,
 * below; 1: the last `plane` entries, above) += recv, except on Dirichlet points of the plane (identity
 * rows on both parts).  recv: device, plane entries of the precision (the neighbour's partial plane of
 * its vmult); y: device, the part's vmult result.  Structured continuous operators only.  Asynchronous.
 * Errors: MFX_EINVAL (null, side not 0 or 1, unknown precision), MFX_EUNSUPPORTED, MFX_ECUDA.
 */
mfx_status mfx_halo_accumulate(const mfx_op* op, mfx_prec prec, int32_t side, const void* recv, void* y,
                               mfx_stream stream);

/*
 * Communication of a partitioned solve, supplied by the caller (NCCL, MPI, a host-side coupler, ...):
 * send[d], recv[d] are caller-owned device buffers of `plane` FP64 entries for side d (0 below, 1
 * above; NULL where the part has no neighbour).  exchange(user): send[d] to the neighbour on side d,
 * its partial plane into recv[d], for every side with a neighbour; called with the stream
 * synchronised, returns 0 on success.  allreduce(user, vals, n): vals[0 .. n) summed over all parts,
 * in place (host doubles), returns 0 on success.  Every part makes the same sequence of calls.
 */
typedef struct {
  void* send[2];
  void* recv[2];
  int32_t (*exchange)(void* user);
  int32_t (*allreduce)(void* user, double* vals, int32_t n);
  void* user;
} mfx_comm;

/*
 * Jacobi-preconditioned CG on the partitioned operator (FP64; the solve of Sec. 6.1 in the distributed
 * form of Sec. 2.6): every vmult is followed by the exchange; the diagonal is exchanged once; each
 * iteration makes two allreduces, (p, Kp) and then (r, z) with (r, r) together, over owned DoFs.  b, x:
 * device FP64, the part's slice of the global vectors (b equal on both copies of a shared DoF); x0 = 0;
 * stopping rule and statuses as mfx_solve (params.tol, params.max_it; other fields ignored).  The host
 * drives the loop (the callbacks are host calls).  Synchronises the stream.
 * Errors: MFX_EINVAL (null, a description that does not match the operator, a missing buffer, a
 * callback that failed), MFX_EUNSUPPORTED (not structured continuous FP64), MFX_ECUDA.
 */
mfx_status mfx_solve_partitioned(const mfx_op* op, const mfx_part_info* part, const mfx_comm* comm, const double* b,
                                 double* x, const mfx_solve_params* params, mfx_solve_stats* stats, mfx_stream stream);

/* ---------------------------------------------------------------- serving */

/*
 * A solve server: a native runtime that admits Poisson solves as they
 * arrive, builds their operators on set-up threads, runs them together in
 * one batch with independent stepping (mfx_batch_advance) on a scheduler
 * thread, and keeps each finished solve's operator and solution on the
 * device until the caller retires it.  Admission: requests wait in a queue
 * and are admitted (policy order) while fewer than max_slots are being set
 * up or solved and the estimated device bytes of all admitted, unretired
 * requests stay within budget_bytes; one request is always admitted when
 * nothing else is, so a request larger than the budget still runs, alone.
 * No counterpart in the paper: this is the serving workload's runtime.
 * All calls are thread-safe; none of them waits for the GPU except
 * mfx_server_result_copy and mfx_server_destroy.
 */
typedef struct mfx_server mfx_server;
enum { MFX_ADMIT_FIFO = 0,            /* arrival order                               */
       MFX_ADMIT_SMALLEST_FIRST = 1 }; /* smallest estimated size first             */
typedef struct {
  int64_t budget_bytes;   /* device bytes for admitted requests (estimate, then exact)     */
  int32_t max_slots;      /* requests in set-up or solving at once (1..4096)                */
  int32_t chunk;          /* inner iterations per scheduler step of a solve (0: 16)         */
  int32_t setup_threads;  /* host threads building operators (0: 4)                        */
  int32_t policy;         /* MFX_ADMIT_*                                                    */
  int32_t reserved[2];
} mfx_server_config;

/*
 * Right-hand side callback, run on a set-up thread once the operator exists:
 * fill b (host, n_dofs doubles, the operator's DoF numbering).  The server
 * copies it to the device and applies mfx_distribute (constrained entries).
 */
typedef void (*mfx_rhs_fn)(const mfx_op* op, double* b, int64_t n_dofs, void* user);

typedef struct {
  /* mesh: either an existing mesh (caller-owned, alive until the request is
     retired) or an octree description (copied at submission; the mesh is
     built on a set-up thread). */
  const mfx_mesh* mesh;
  int32_t nx, ny, nz, reserved0;   /* octree: coarse cells per direction        */
  const int32_t* leaves;           /* octree: n_leaves x 4 (level, i, j, k)      */
  int64_t n_leaves;
  const double* coarse_vertices;   /* octree: NULL = unit cube (copied)          */
  mfx_op_desc desc;                /* degree, coefficient, precisions (need both for mixed) */
  mfx_solve_params params;         /* tol, mixed, preconditioner, ...            */
  mfx_rhs_fn rhs;                  /* NULL: b = 1 on every DoF before distribute */
  void* user;
  int64_t est_bytes;               /* 0: estimated from cells and degree         */
} mfx_request;

enum { MFX_REQ_QUEUED = 0, MFX_REQ_SETUP = 1, MFX_REQ_RUNNING = 2, MFX_REQ_DONE = 3,
       MFX_REQ_CANCELLED = 4, MFX_REQ_FAILED = 5 };

typedef struct {
  int32_t state;                   /* MFX_REQ_*                                  */
  int32_t error;                   /* failed: the mfx_status of the failing call */
  int64_t n_dofs;
  int64_t bytes;                   /* device bytes held (estimate until set up)  */
  double t_submit, t_admit, t_ready, t_done;  /* seconds since the server was created (-1: not yet) */
  double setup_seconds;            /* set-up thread time (mesh, operator, workspace, rhs) */
  mfx_solve_stats stats;           /* final solve statistics (state DONE)        */
} mfx_request_info;

typedef struct {
  int64_t submitted, queued, in_setup, running, done, cancelled, failed, retired;
  int64_t bytes_in_use;            /* admitted, not yet retired                  */
  int32_t max_concurrent;          /* most solves running at once so far         */
  int32_t reserved;
  double now;                      /* seconds since creation                     */
} mfx_server_stats;

/* The mfx_server_* calls have no counterpart in the paper (see above); each request's solve is
 * that of mfx_solve (Sec. 6.1) on an octree mesh with hanging nodes (Sec. 3.3).
 * Errors: MFX_EINVAL (bad config), MFX_ENOMEM, MFX_ECUDA. */
mfx_status mfx_server_create(mfx_server** out, const mfx_server_config* config);
/* Cancels what is queued, waits for running and set-up work, frees everything. */
void mfx_server_destroy(mfx_server* server);
/* Queue a request; ticket identifies it.  Errors: MFX_EINVAL (no mesh, bad description). */
mfx_status mfx_server_submit(mfx_server* server, const mfx_request* request, int64_t* ticket);
/* Current state and times of a request.  Errors: MFX_EINVAL (unknown or retired ticket). */
mfx_status mfx_server_poll(mfx_server* server, int64_t ticket, mfx_request_info* info);
/* Cancel: a queued request is dropped at once; one in set-up or running is stopped at the
 * scheduler's next step (state MFX_REQ_CANCELLED).  Finished requests are left as they are. */
mfx_status mfx_server_cancel(mfx_server* server, int64_t ticket);
/* Copy the solution of a DONE request to host memory (n = n_dofs doubles).  Errors: MFX_EINVAL
 * (unknown ticket, wrong n), MFX_EBUSY (not done). */
mfx_status mfx_server_result_copy(mfx_server* server, int64_t ticket, double* x_host, int64_t n);
/* The operator of a DONE request (valid until retired), e.g. to apply it to the solution. */
mfx_status mfx_server_operator(mfx_server* server, int64_t ticket, const mfx_op** op);
/* Free a finished (done, cancelled or failed) request's device data and forget the ticket.
 * Errors: MFX_EINVAL (unknown ticket), MFX_EBUSY (still queued, in set-up or running). */
mfx_status mfx_server_retire(mfx_server* server, int64_t ticket);
/* Counters of the server so far.  Errors: MFX_EINVAL (null argument). */
mfx_status mfx_server_stats_get(mfx_server* server, mfx_server_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* MFX_H */
