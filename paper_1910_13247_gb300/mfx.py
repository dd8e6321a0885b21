"""Thin ctypes binding of libmfx.so (argument marshalling only).

Every computation runs in the CUDA library; tensors are passed by device
pointer and streams by handle (PyTorch provides memory and streams only).
If the library is missing, loading raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmfx.so")

F64, F32 = 0, 1
COEF_CONSTANT, COEF_TRIG, COEF_QPOINT, COEF_FUNCTION = 0, 1, 2, 3
CONTINUOUS, SIPG = 0, 1  # discretization of an operator (mfx_op_desc.discretization)
# FP32 vmult kernel of a structured operator at k = 1..4 (mfx_op_desc.structured_kernel)
KERNEL_AUTO, KERNEL_TEN_PHASE, KERNEL_FIVE_PHASE, KERNEL_FIVE_PHASE_STAGED = 0, 1, 2, 3
PRECOND_JACOBI, PRECOND_CHEBYSHEV = 0, 1
OK, EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, EMESH, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
NOT_CONVERGED, BREAKDOWN = 1, 2
FACE_X0, FACE_X1, FACE_Y0, FACE_Y1, FACE_Z0, FACE_Z1, FACES_ALL = 1, 2, 4, 8, 16, 32, 63


class MfxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mfx error {code}: {msg}")
        self.code = code


POINT_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)
MAP_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def point_fn(f):
    """Wrap f(x, y, z) -> float as an mfx_point_fn (keep the result alive while the library may call it)."""
    return POINT_FN(lambda x, _user: float(f(x[0], x[1], x[2])))


class OpDesc(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("n_q_1d", ctypes.c_int32), ("coef_kind", ctypes.c_int32),
                ("precisions", ctypes.c_int32), ("coef_par", ctypes.c_double * 2),
                ("coef_qpoint", ctypes.c_void_p), ("cells_per_block", ctypes.c_int32),
                ("discretization", ctypes.c_int32), ("coef_fn", POINT_FN), ("coef_user", ctypes.c_void_p),
                ("dg_penalty", ctypes.c_double), ("structured_kernel", ctypes.c_int32)]


class OpInfo(ctypes.Structure):
    _fields_ = [("n_dofs", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_constrained", ctypes.c_int64),
                ("n_masters", ctypes.c_int64), ("n_hanging", ctypes.c_int64), ("bytes_device", ctypes.c_int64),
                ("degree", ctypes.c_int32), ("n_q_1d", ctypes.c_int32), ("structured", ctypes.c_int32),
                ("cells_per_block", ctypes.c_int32), ("discretization", ctypes.c_int32),
                ("structured_kernel", ctypes.c_int32), ("box_metric", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_it", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("cheb_degree", ctypes.c_int32), ("mixed", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("lanczos_start", ctypes.c_void_p), ("inner_max_it", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("inner_iterations", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class PartInfo(ctypes.Structure):
    _fields_ = [("cz0", ctypes.c_int32), ("nz", ctypes.c_int32), ("dirichlet", ctypes.c_uint32),
                ("has_lo", ctypes.c_int32), ("has_hi", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dof0", ctypes.c_int64), ("n_dofs", ctypes.c_int64), ("n_owned", ctypes.c_int64),
                ("plane", ctypes.c_int64), ("vertex0", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32)


class Comm(ctypes.Structure):
    _fields_ = [("send", ctypes.c_void_p * 2), ("recv", ctypes.c_void_p * 2), ("exchange", EXCHANGE_FN),
                ("allreduce", ALLREDUCE_FN), ("user", ctypes.c_void_p)]


class MgParams(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_int32), ("smoother_degree", ctypes.c_int32),
                ("smoothing_range", ctypes.c_double), ("lanczos_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("setup_threads", ctypes.c_int32), ("policy", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p)


class Request(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("leaves", ctypes.c_void_p), ("n_leaves", ctypes.c_int64),
                ("coarse_vertices", ctypes.c_void_p), ("desc", OpDesc), ("params", SolveParams),
                ("rhs", RHS_FN), ("user", ctypes.c_void_p), ("est_bytes", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("n_dofs", ctypes.c_int64),
                ("bytes", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_ready", ctypes.c_double), ("t_done", ctypes.c_double), ("setup_seconds", ctypes.c_double),
                ("stats", SolveStats)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("queued", ctypes.c_int64), ("in_setup", ctypes.c_int64),
                ("running", ctypes.c_int64), ("done", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("retired", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("max_concurrent", ctypes.c_int32), ("reserved", ctypes.c_int32), ("now", ctypes.c_double)]


class IndexTables(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("nodes_1d", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_dofs", ctypes.c_int64), ("n_rows", ctypes.c_int64), ("n_masters", ctypes.c_int64),
                ("n_hdofs", ctypes.c_int64), ("cell_dofs", ctypes.c_void_p), ("cptr", ctypes.c_void_p),
                ("cmaster", ctypes.c_void_p), ("hface", ctypes.c_void_p), ("hedge", ctypes.c_void_p),
                ("hoff", ctypes.c_void_p), ("hdofs", ctypes.c_void_p), ("cell_list", ctypes.c_void_p * 2),
                ("n_list", ctypes.c_int64 * 2)]


ADMIT_FIFO, ADMIT_SMALLEST_FIRST = 0, 1
REQ_QUEUED, REQ_SETUP, REQ_RUNNING, REQ_DONE, REQ_CANCELLED, REQ_FAILED = range(6)

_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load libmfx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1910_13247_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int32
    sig = {
        "mfx_last_error": (ctypes.c_char_p, []),
        "mfx_version": (ctypes.c_char_p, []),
        "mfx_mesh_create_structured": (S, [ctypes.POINTER(_VP), S, S, S, _VP]),
        "mfx_mesh_create_octree": (S, [ctypes.POINTER(_VP), S, S, S, _VP, _VP, ctypes.c_int64]),
        "mfx_mesh_destroy": (None, [_VP]),
        "mfx_mesh_transform": (S, [_VP, MAP_FN, _VP]),
        "mfx_mesh_set_dirichlet": (S, [_VP, ctypes.c_uint32]),
        "mfx_mesh_get_dirichlet": (S, [_VP, ctypes.POINTER(ctypes.c_uint32)]),
        "mfx_rhs_function": (S, [_VP, POINT_FN, _VP, _VP, _VP]),
        "mfx_mesh_table_sizes": (S, [_VP, S, _VP, _VP, _VP, _VP]),
        "mfx_mesh_tables": (S, [_VP, S, _VP, _VP, _VP, _VP, _VP]),
        "mfx_mesh_hanging_tables": (S, [_VP, S, _VP, _VP, _VP, _VP, _VP]),
        "mfx_operator_create": (S, [ctypes.POINTER(_VP), _VP, ctypes.POINTER(OpDesc), _VP]),
        "mfx_operator_destroy": (None, [_VP]),
        "mfx_operator_release": (S, [_VP, _VP]),
        "mfx_solver_prepare": (S, [_VP]),
        "mfx_operator_info": (S, [_VP, ctypes.POINTER(OpInfo)]),
        "mfx_get_tables": (S, [_VP, _VP, _VP, _VP, _VP, _VP]),
        "mfx_vmult": (S, [_VP, S, _VP, _VP, _VP]),
        "mfx_vmult_host": (S, [_VP, S, S, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
        "mfx_diagonal": (S, [_VP, S, _VP, _VP]),
        "mfx_device_check": (S, [_VP, _VP]),
        "mfx_selftest_bounded_wait": (S, [_VP, _VP]),
        "mfx_validate_tables": (S, [_VP, _VP, _VP]),
        "mfx_operator_validate": (S, [_VP, _VP, _VP]),
        "mfx_quadrature_points": (S, [_VP, _VP, _VP]),
        "mfx_rhs": (S, [_VP, _VP, _VP, _VP]),
        "mfx_distribute": (S, [_VP, _VP, _VP]),
        "mfx_dot": (S, [_VP, S, ctypes.c_int64, _VP, _VP, _VP, _VP]),
        "mfx_dot_noalloc": (S, [S, ctypes.c_int64, _VP, _VP, _VP, _VP]),
        "mfx_chebyshev": (S, [_VP, S, _VP, _VP, S, ctypes.c_double, ctypes.c_double, _VP]),
        "mfx_solve_params_default": (None, [ctypes.POINTER(SolveParams)]),
        "mfx_solve": (S, [_VP, _VP, _VP, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _VP]),
        "mfx_batch_create": (S, [ctypes.POINTER(_VP), S, S]),
        "mfx_batch_destroy": (None, [_VP]),
        "mfx_batch_add": (S, [_VP, _VP, _VP, _VP, ctypes.POINTER(SolveParams), ctypes.POINTER(S)]),
        "mfx_batch_step": (S, [_VP, ctypes.POINTER(S)]),
        "mfx_batch_advance": (S, [_VP, ctypes.POINTER(S)]),
        "mfx_batch_poll": (S, [_VP, S, ctypes.POINTER(S), ctypes.POINTER(SolveStats)]),
        "mfx_batch_run": (S, [_VP, ctypes.POINTER(S)]),
        "mfx_batch_release": (S, [_VP, S]),
        "mfx_mg_params_default": (None, [ctypes.POINTER(MgParams)]),
        "mfx_mg_create": (S, [ctypes.POINTER(_VP), _VP, ctypes.POINTER(OpDesc), ctypes.POINTER(MgParams), _VP]),
        "mfx_mg_destroy": (None, [_VP]),
        "mfx_mg_info": (S, [_VP, ctypes.POINTER(S), ctypes.POINTER(S)]),
        "mfx_mg_operator": (_VP, [_VP, S]),
        "mfx_mg_get_bounds": (S, [_VP, S, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "mfx_mg_set_bounds": (S, [_VP, S, ctypes.c_double, ctypes.c_double]),
        "mfx_mg_vcycle": (S, [_VP, S, _VP, _VP, _VP]),
        "mfx_mg_solve": (S, [_VP, _VP, _VP, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _VP]),
        "mfx_partition_box": (S, [S, S, S, S, ctypes.c_uint32, S, S, ctypes.POINTER(PartInfo)]),
        "mfx_halo_accumulate": (S, [_VP, S, S, _VP, _VP, _VP]),
        "mfx_solve_partitioned": (S, [_VP, ctypes.POINTER(PartInfo), ctypes.POINTER(Comm), _VP, _VP,
                                      ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _VP]),
        "mfx_server_create": (S, [ctypes.POINTER(_VP), ctypes.POINTER(ServerConfig)]),
        "mfx_server_destroy": (None, [_VP]),
        "mfx_server_submit": (S, [_VP, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
        "mfx_server_poll": (S, [_VP, ctypes.c_int64, ctypes.POINTER(RequestInfo)]),
        "mfx_server_cancel": (S, [_VP, ctypes.c_int64]),
        "mfx_server_result_copy": (S, [_VP, ctypes.c_int64, _VP, ctypes.c_int64]),
        "mfx_server_operator": (S, [_VP, ctypes.c_int64, ctypes.POINTER(_VP)]),
        "mfx_server_retire": (S, [_VP, ctypes.c_int64]),
        "mfx_server_stats_get": (S, [_VP, ctypes.POINTER(ServerStats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(code):
    if code < 0:
        raise MfxError(code, lib().mfx_last_error().decode())
    return code


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("vectors must be float64 or float32")


def partition_box(nx, ny, nz, degree, n_parts, part, dirichlet=0x3F):
    """The slab of cells along z that part `part` of n_parts takes, and its DoF bookkeeping (host-only,
    mfx_partition_box): a dict with cz0, nz, dirichlet, has_lo, has_hi, dof0, n_dofs, n_owned, plane,
    vertex0."""
    info = PartInfo()
    check(lib().mfx_partition_box(nx, ny, nz, degree, dirichlet, n_parts, part, ctypes.byref(info)))
    return info


def halo_accumulate(op, side, recv, y, stream=None):
    """y's shared plane on `side` (0 below, 1 above) += recv, except on Dirichlet points (mfx_halo_accumulate)."""
    check(lib().mfx_halo_accumulate(op.handle, _prec_of(y), side, _ptr(recv), _ptr(y), _stream(stream)))


def solve_partitioned(op, part, b, x, exchange, allreduce, send, recv, tol=1e-10, max_it=100000, stream=None):
    """Jacobi-PCG on a partitioned operator (mfx_solve_partitioned).  part: the PartInfo of this part;
    send, recv: two device FP64 tensors each (or None where the part has no neighbour), `plane` entries;
    exchange(): send to the neighbours, fill recv; allreduce(list of floats) -> list of floats summed over
    the parts.  Returns the solve statistics."""
    c = Comm()
    for d in range(2):
        c.send[d] = send[d].data_ptr() if send[d] is not None else None
        c.recv[d] = recv[d].data_ptr() if recv[d] is not None else None

    def _ex(_user):
        try:
            exchange()
            return 0
        except Exception:  # reported to the library as a failed callback
            import traceback
            traceback.print_exc()
            return 1

    def _ar(_user, vals, n):
        try:
            out = allreduce([vals[i] for i in range(n)])
            for i in range(n):
                vals[i] = float(out[i])
            return 0
        except Exception:
            import traceback
            traceback.print_exc()
            return 1

    c.exchange = EXCHANGE_FN(_ex)
    c.allreduce = ALLREDUCE_FN(_ar)
    p = make_params(tol=tol, max_it=max_it)
    st = SolveStats()
    rc = lib().mfx_solve_partitioned(op.handle, ctypes.byref(part), ctypes.byref(c), _ptr(b), _ptr(x), ctypes.byref(p),
                                     ctypes.byref(st), _stream(stream))
    if rc < 0:
        check(rc)
    return st.as_dict()


def dot_noalloc(a, b, out, n=None, stream=None):
    """out[0] = sum a_i b_i (FP64) without any device allocation (fixed library scratch)."""
    n = a.numel() if n is None else n
    check(lib().mfx_dot_noalloc(_prec_of(a), n, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))
    return out


class Mesh:
    """Host mesh description (structured box or octree)."""

    def __init__(self, handle, structured):
        self.handle = handle
        self.structured = structured

    @classmethod
    def structured_box(cls, nx, ny, nz, vertices=None, dirichlet=FACES_ALL):
        h = ctypes.c_void_p()
        v = None
        if vertices is not None:
            v = np.ascontiguousarray(vertices, dtype=np.float64)
            assert v.size == 3 * (nx + 1) * (ny + 1) * (nz + 1)
        check(lib().mfx_mesh_create_structured(ctypes.byref(h), nx, ny, nz,
                                               v.ctypes.data_as(_VP) if v is not None else None))
        return cls(h, True).set_dirichlet(dirichlet)

    @classmethod
    def octree(cls, nx, ny, nz, leaves, coarse_vertices=None, dirichlet=FACES_ALL):
        h = ctypes.c_void_p()
        lv = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1, 4)
        v = None if coarse_vertices is None else np.ascontiguousarray(coarse_vertices, dtype=np.float64)
        check(lib().mfx_mesh_create_octree(ctypes.byref(h), nx, ny, nz,
                                           v.ctypes.data_as(_VP) if v is not None else None,
                                           lv.ctypes.data_as(_VP), lv.shape[0]))
        return cls(h, False).set_dirichlet(dirichlet)

    def set_dirichlet(self, faces):
        """Dirichlet faces as a bit mask (FACE_X0 | FACE_X1 | ...); the others are natural boundaries."""
        check(lib().mfx_mesh_set_dirichlet(self.handle, faces))
        return self

    def dirichlet(self):
        f = ctypes.c_uint32()
        check(lib().mfx_mesh_get_dirichlet(self.handle, ctypes.byref(f)))
        return f.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfx_mesh_destroy(self.handle)
            self.handle = None

    def transform(self, phi):
        """Move every (coarse) vertex v to phi(x, y, z) -> (x', y', z'), on the host (mfx_mesh_transform)."""
        def call(inp, out, _user):
            out[0], out[1], out[2] = phi(inp[0], inp[1], inp[2])
        check(lib().mfx_mesh_transform(self.handle, MAP_FN(call), None))
        return self

    def tables(self, degree):
        """DoF and constraint tables at degree k, computed on the host (no GPU needed)."""
        c, n, nc, nm = (ctypes.c_int64() for _ in range(4))
        check(lib().mfx_mesh_table_sizes(self.handle, degree, ctypes.byref(c), ctypes.byref(n),
                                         ctypes.byref(nc), ctypes.byref(nm)))
        n3 = (degree + 1) ** 3
        cd = np.zeros(c.value * n3, dtype=np.int32)
        co = np.zeros(nc.value, dtype=np.int32)
        cp = np.zeros(nc.value + 1, dtype=np.int64)
        cm = np.zeros(max(1, nm.value), dtype=np.int32)
        cw = np.zeros(max(1, nm.value), dtype=np.float64)
        check(lib().mfx_mesh_tables(self.handle, degree, cd.ctypes.data_as(_VP), co.ctypes.data_as(_VP),
                                    cp.ctypes.data_as(_VP), cm.ctypes.data_as(_VP), cw.ctypes.data_as(_VP)))
        return {"n_dofs": n.value, "cell_dofs": cd.reshape(c.value, n3), "constrained": co, "cptr": cp,
                "cmaster": cm[:nm.value], "cweight": cw[:nm.value]}

    def hanging_tables(self, degree):
        """Tensor-product form of the hanging-node constraints at degree k, computed on the host: per cell
        the hanging-face word, the hanging-edge word and the offset of its coarse DoFs in `hdofs`."""
        c, nh = ctypes.c_int64(), ctypes.c_int64()
        check(lib().mfx_mesh_table_sizes(self.handle, degree, ctypes.byref(c), None, None, None))
        check(lib().mfx_mesh_hanging_tables(self.handle, degree, None, None, None, None, ctypes.byref(nh)))
        hf = np.zeros(c.value, dtype=np.uint32)
        he = np.zeros(c.value, dtype=np.uint32)
        ho = np.zeros(c.value, dtype=np.int64)
        hd = np.zeros(max(1, nh.value), dtype=np.int32)
        check(lib().mfx_mesh_hanging_tables(self.handle, degree, hf.ctypes.data_as(_VP), he.ctypes.data_as(_VP),
                                            ho.ctypes.data_as(_VP), hd.ctypes.data_as(_VP), ctypes.byref(nh)))
        return {"hface": hf, "hedge": he, "hoff": ho, "hdofs": hd[:nh.value]}


class Operator:
    """The condensed Q_k operator of one mesh (geometry and tables on the device)."""

    def __init__(self, mesh, degree, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), precisions=3,
                 coef_qpoint=None, stream=None, cells_per_block=0, coef_fn=None, discretization=CONTINUOUS,
                 dg_penalty=1.0, structured_kernel=KERNEL_AUTO):
        """discretization=SIPG: the symmetric interior penalty DG operator (uniform box, constant
        coefficient coef_par[0], penalty eta = dg_penalty, cell-major DoFs).  structured_kernel: the
        FP32 vmult kernel of a structured operator at k = 1..4 (KERNEL_*; KERNEL_AUTO: timed)."""
        d = OpDesc()
        if coef_fn is not None:  # a(x, y, z) on the host at every quadrature point
            coef_kind = COEF_FUNCTION
            d.coef_fn = point_fn(coef_fn)
        d.degree = degree
        d.n_q_1d = 0
        d.coef_kind = coef_kind
        d.precisions = precisions
        d.coef_par[0], d.coef_par[1] = coef_par
        d.coef_qpoint = coef_qpoint.data_ptr() if coef_qpoint is not None else None
        d.cells_per_block = cells_per_block
        d.discretization = discretization
        d.dg_penalty = dg_penalty
        d.structured_kernel = structured_kernel
        h = ctypes.c_void_p()
        check(lib().mfx_operator_create(ctypes.byref(h), mesh.handle, ctypes.byref(d), _stream(stream)))
        self.handle = h
        self.degree = degree
        self._info = self.info()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfx_operator_destroy(self.handle)
            self.handle = None

    def release(self, stream=None):
        """Free the operator in stream order on `stream`, without a device-wide wait; every use of the
        operator must already be complete or ordered before that stream (mfx_operator_release)."""
        if getattr(self, "handle", None):
            h, self.handle = self.handle, None
            check(lib().mfx_operator_release(h, _stream(stream)))

    def prepare_solver(self):
        """Allocate the solver workspace now rather than at the first solve (mfx_solver_prepare)."""
        check(lib().mfx_solver_prepare(self.handle))
        self._info = self.info()
        return self

    def info(self):
        i = OpInfo()
        check(lib().mfx_operator_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    @property
    def n_dofs(self):
        return self._info["n_dofs"]

    @property
    def n_cells(self):
        return self._info["n_cells"]

    def tables(self):
        i = self.info()
        n3 = (self.degree + 1) ** 3
        cd = np.zeros(i["n_cells"] * n3, dtype=np.int32)
        co = np.zeros(i["n_constrained"], dtype=np.int32)
        cp = np.zeros(i["n_constrained"] + 1, dtype=np.int64)
        cm = np.zeros(max(1, i["n_masters"]), dtype=np.int32)
        cw = np.zeros(max(1, i["n_masters"]), dtype=np.float64)
        check(lib().mfx_get_tables(self.handle, cd.ctypes.data_as(_VP), co.ctypes.data_as(_VP),
                                   cp.ctypes.data_as(_VP), cm.ctypes.data_as(_VP), cw.ctypes.data_as(_VP)))
        return {"cell_dofs": cd.reshape(i["n_cells"], n3), "constrained": co, "cptr": cp,
                "cmaster": cm[:i["n_masters"]], "cweight": cw[:i["n_masters"]]}

    def vmult(self, src, dst, stream=None):
        assert src.is_cuda and dst.is_cuda and src.dtype == dst.dtype and src.is_contiguous() and dst.is_contiguous()
        assert src.numel() == self.n_dofs and dst.numel() == self.n_dofs
        check(lib().mfx_vmult(self.handle, _prec_of(src), _ptr(src), _ptr(dst), _stream(stream)))
        return dst

    def vmult_host(self, srcs, dsts, stream=None):
        """dst[i] = K src[i] for host vectors (CPU tensors, pinned for full speed), pipelined through the
        device (mfx_vmult_host); returns when every result is in host memory."""
        assert len(srcs) == len(dsts) and len(srcs) > 0
        dt = srcs[0].dtype
        for t in list(srcs) + list(dsts):
            assert (not t.is_cuda) and t.dtype == dt and t.is_contiguous() and t.numel() == self.n_dofs
        n = len(srcs)
        sp = (_VP * n)(*[t.data_ptr() for t in srcs])
        dp = (_VP * n)(*[t.data_ptr() for t in dsts])
        check(lib().mfx_vmult_host(self.handle, _prec_of(srcs[0]), n, sp, dp, _stream(stream)))
        return dsts

    def device_check(self):
        """Synchronise and raise if a bounded device wait of this operator ran out."""
        check(lib().mfx_device_check(self.handle, _stream()))

    def validate(self):
        """Checked mode: count, on the device, the entries of this operator's index tables that are out of
        range or inconsistent (mfx_operator_validate); 0 for sound tables."""
        nb = ctypes.c_int64()
        code = lib().mfx_operator_validate(self.handle, ctypes.byref(nb), _stream())
        if code != EMESH:
            check(code)
        return nb.value

    def selftest_bounded_wait(self):
        """Launch a kernel whose bounded wait runs out (about one second); the next device_check raises
        MfxError with code ETIMEOUT."""
        check(lib().mfx_selftest_bounded_wait(self.handle, _stream()))

    def diagonal(self, out):
        assert out.numel() == self.n_dofs
        check(lib().mfx_diagonal(self.handle, _prec_of(out), _ptr(out), _stream()))
        return out

    def quadrature_points(self, out):
        n3 = (self.degree + 1) ** 3
        assert out.numel() == self.n_cells * n3 * 3 and out.dtype.itemsize == 8
        check(lib().mfx_quadrature_points(self.handle, _ptr(out), _stream()))
        return out

    def rhs(self, fq, b):
        check(lib().mfx_rhs(self.handle, _ptr(fq), _ptr(b), _stream()))
        return b

    def rhs_function(self, f, b):
        """Load vector of a host function f(x, y, z), evaluated at the quadrature points (mfx_rhs_function)."""
        check(lib().mfx_rhs_function(self.handle, point_fn(f), None, _ptr(b), _stream()))
        return b

    def distribute(self, x, stream=None):
        check(lib().mfx_distribute(self.handle, _ptr(x), _stream(stream)))
        return x

    def dot(self, a, b, out):
        check(lib().mfx_dot(self.handle, _prec_of(a), a.numel(), _ptr(a), _ptr(b), _ptr(out), _stream()))
        return out

    def chebyshev(self, r, z, degree, lo, hi):
        check(lib().mfx_chebyshev(self.handle, _prec_of(r), _ptr(r), _ptr(z), degree, lo, hi, _stream()))
        return z

    def solve_params(self, **kw):
        return make_params(**kw)

    def solve(self, b, x, tol=1e-10, max_it=100000, precond=PRECOND_JACOBI, cheb_degree=5, mixed=False,
              inner_tol=1e-4, check_every=0, lanczos_steps=15, cheb_lo=0.0, cheb_hi=0.0, lanczos_start=None,
              inner_max_it=10000):
        p = SolveParams()
        lib().mfx_solve_params_default(ctypes.byref(p))
        p.tol, p.max_it, p.precond, p.cheb_degree = tol, max_it, precond, cheb_degree
        p.mixed, p.inner_tol, p.check_every, p.lanczos_steps = int(mixed), inner_tol, check_every, lanczos_steps
        p.cheb_lo, p.cheb_hi = cheb_lo, cheb_hi
        p.lanczos_start = lanczos_start.data_ptr() if lanczos_start is not None else None
        p.inner_max_it = inner_max_it
        st = SolveStats()
        check(lib().mfx_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(st), _stream()))
        return st.as_dict()


def validate_tables(n_cells, nodes_1d, n_dofs, cell_dofs, n_rows=0, cptr=None, cmaster=None, hface=None,
                    hedge=None, hoff=None, hdofs=None, cell_lists=(), stream=None):
    """Checked mode on caller-supplied device tables (torch tensors; mfx_validate_tables): returns the number
    of entries out of range or inconsistent."""
    t = IndexTables()
    t.n_cells, t.nodes_1d, t.n_dofs, t.n_rows = n_cells, nodes_1d, n_dofs, n_rows
    t.n_masters = cmaster.numel() if cmaster is not None else 0
    t.n_hdofs = hdofs.numel() if hdofs is not None else 0
    for name, v in (("cell_dofs", cell_dofs), ("cptr", cptr), ("cmaster", cmaster), ("hface", hface),
                    ("hedge", hedge), ("hoff", hoff), ("hdofs", hdofs)):
        setattr(t, name, v.data_ptr() if v is not None else None)
    for i, lst in enumerate(cell_lists):
        t.cell_list[i], t.n_list[i] = lst.data_ptr(), lst.numel()
    nb = ctypes.c_int64()
    code = lib().mfx_validate_tables(ctypes.byref(t), ctypes.byref(nb), _stream(stream))
    if code != EMESH:
        check(code)
    return nb.value


def make_params(tol=1e-10, max_it=100000, precond=PRECOND_JACOBI, cheb_degree=5, mixed=False, inner_tol=1e-4,
                check_every=0, lanczos_steps=15, cheb_lo=0.0, cheb_hi=0.0, lanczos_start=None, inner_max_it=10000):
    p = SolveParams()
    lib().mfx_solve_params_default(ctypes.byref(p))
    p.tol, p.max_it, p.precond, p.cheb_degree = tol, max_it, precond, cheb_degree
    p.mixed, p.inner_tol, p.check_every, p.lanczos_steps = int(mixed), inner_tol, check_every, lanczos_steps
    p.cheb_lo, p.cheb_hi = cheb_lo, cheb_hi
    p.lanczos_start = lanczos_start.data_ptr() if lanczos_start is not None else None
    p.inner_max_it = inner_max_it
    return p


class Batch:
    """Slots of independent solves advanced together, one graph launch per tick (mfx_batch_*)."""

    def __init__(self, max_slots, chunk=8):
        h = ctypes.c_void_p()
        check(lib().mfx_batch_create(ctypes.byref(h), max_slots, chunk))
        self.handle = h
        self._keep = {}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfx_batch_destroy(self.handle)
            self.handle = None

    def add(self, op, b, x, **kw):
        p = make_params(**kw)
        slot = ctypes.c_int32()
        check(lib().mfx_batch_add(self.handle, op.handle, _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(slot)))
        self._keep[slot.value] = (op, b, x)
        return slot.value

    def step(self):
        n = ctypes.c_int32()
        check(lib().mfx_batch_step(self.handle, ctypes.byref(n)))
        return n.value

    def advance(self):
        """Independent stepping: each finished slot takes its next step; returns active slots."""
        n = ctypes.c_int32()
        check(lib().mfx_batch_advance(self.handle, ctypes.byref(n)))
        return n.value

    def poll(self, slot):
        done = ctypes.c_int32()
        st = SolveStats()
        check(lib().mfx_batch_poll(self.handle, slot, ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), st.as_dict()

    def release(self, slot):
        check(lib().mfx_batch_release(self.handle, slot))
        self._keep.pop(slot, None)

    def run(self, max_ticks=1000000):
        """Host-driven ticks (mfx_batch_step) until every slot is done; returns the ticks."""
        ticks = 0
        while self.step() > 0 and ticks < max_ticks:
            ticks += 1
        return ticks

    def run_once(self):
        """Every active slot's whole solve in one graph launch, the device deciding when each problem
        stops (mfx_batch_run); returns the number of slots run."""
        n = ctypes.c_int32()
        check(lib().mfx_batch_run(self.handle, ctypes.byref(n)))
        return n.value


class Server:
    """Native solve server (mfx_server_*): admission by memory budget, operator set-up on library threads,
    a scheduler thread stepping every running solve.  Requests carry an octree description (or a Mesh) and
    an optional right-hand side function rhs(n_dofs) -> array of n_dofs values (called on a set-up thread)."""

    def __init__(self, budget_bytes=64 << 30, max_slots=32, chunk=16, setup_threads=4, policy=ADMIT_FIFO):
        c = ServerConfig()
        c.budget_bytes, c.max_slots, c.chunk, c.setup_threads, c.policy = budget_bytes, max_slots, chunk, \
            setup_threads, policy
        h = ctypes.c_void_p()
        check(lib().mfx_server_create(ctypes.byref(h), ctypes.byref(c)))
        self.handle = h
        self._keep = {}  # ticket -> objects the library may still use (mesh, callback)

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfx_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        self.close()

    def submit(self, degree, leaves=None, n_coarse=None, mesh=None, rhs=None, tol=1e-10, mixed=True,
               coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), est_bytes=0, **params):
        r = Request()
        keep = []
        if mesh is not None:
            r.mesh = mesh.handle
            keep.append(mesh)
        else:
            lv = np.ascontiguousarray(leaves, dtype=np.int32)
            nx, ny, nz = n_coarse if isinstance(n_coarse, (tuple, list)) else (n_coarse,) * 3
            r.nx, r.ny, r.nz = nx, ny, nz
            r.leaves = lv.ctypes.data_as(_VP)
            r.n_leaves = lv.shape[0]
            keep.append(lv)  # copied by the library at submission; kept only for the call
        r.desc.degree, r.desc.coef_kind, r.desc.precisions = degree, coef_kind, 3
        r.desc.coef_par[0], r.desc.coef_par[1] = coef_par
        r.params = make_params(tol=tol, mixed=mixed, **params)
        if rhs is not None:
            def fill(_op, b, n, _user):
                np.ctypeslib.as_array(b, shape=(n,))[:] = rhs(n)
            cb = RHS_FN(fill)
            r.rhs = cb
            keep.append(cb)
        r.est_bytes = est_bytes
        t = ctypes.c_int64()
        check(lib().mfx_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket):
        i = RequestInfo()
        check(lib().mfx_server_poll(self.handle, ticket, ctypes.byref(i)))
        d = {f: getattr(i, f) for f, _ in i._fields_ if f != "stats"}
        d["stats"] = i.stats.as_dict()
        return d

    def cancel(self, ticket):
        check(lib().mfx_server_cancel(self.handle, ticket))

    def result(self, ticket):
        n = self.poll(ticket)["n_dofs"]
        x = np.empty(n, dtype=np.float64)
        check(lib().mfx_server_result_copy(self.handle, ticket, x.ctypes.data_as(_VP), n))
        return x

    def retire(self, ticket):
        check(lib().mfx_server_retire(self.handle, ticket))
        self._keep.pop(ticket, None)

    def stats(self):
        st = ServerStats()
        check(lib().mfx_server_stats_get(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}


class Multigrid:
    """Geometric multigrid hierarchy of a structured mesh (mfx_mg_*): level operators, transfers,
    Chebyshev smoothers, exact coarse solve; V-cycle application and MG-preconditioned solves."""

    def __init__(self, mesh, degree, coef_kind=COEF_CONSTANT, coef_par=(1.0, 0.0), max_levels=0,
                 smoother_degree=6, smoothing_range=20.0, lanczos_steps=15, stream=None, discretization=CONTINUOUS,
                 dg_penalty=1.0):
        """discretization=SIPG: the SIPG operator on top of the continuous hierarchy of the same mesh."""
        d = OpDesc()
        d.degree, d.n_q_1d, d.coef_kind, d.precisions = degree, 0, coef_kind, 3
        d.discretization, d.dg_penalty = discretization, dg_penalty
        d.coef_par[0], d.coef_par[1] = coef_par
        p = MgParams()
        lib().mfx_mg_params_default(ctypes.byref(p))
        p.max_levels, p.smoother_degree, p.smoothing_range, p.lanczos_steps = max_levels, smoother_degree, \
            smoothing_range, lanczos_steps
        h = ctypes.c_void_p()
        check(lib().mfx_mg_create(ctypes.byref(h), mesh.handle, ctypes.byref(d), ctypes.byref(p), _stream(stream)))
        self.handle = h
        self.degree = degree
        nl, nf = ctypes.c_int32(), ctypes.c_int32()
        check(lib().mfx_mg_info(h, ctypes.byref(nl), ctypes.byref(nf)))
        self.n_levels, self.coarse_free_dofs = nl.value, nf.value

    @property
    def fine(self):
        """The finest level's operator (a view that keeps the hierarchy alive)."""
        return self.operator(self.n_levels - 1)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mfx_mg_destroy(self.handle)
            self.handle = None

    def operator(self, level):
        """Non-owning view of a level's operator (0 = coarsest)."""
        h = lib().mfx_mg_operator(self.handle, level)
        if not h:
            raise MfxError(EINVAL, "bad level")
        h = ctypes.c_void_p(h)
        i = OpInfo()
        check(lib().mfx_operator_info(h, ctypes.byref(i)))
        return _OpView(h, self.degree, {f: getattr(i, f) for f, _ in i._fields_}, self)

    def bounds(self, level):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        check(lib().mfx_mg_get_bounds(self.handle, level, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def set_bounds(self, level, lo, hi):
        check(lib().mfx_mg_set_bounds(self.handle, level, lo, hi))

    def vcycle(self, r, z, stream=None):
        check(lib().mfx_mg_vcycle(self.handle, _prec_of(r), _ptr(r), _ptr(z), _stream(stream)))
        return z

    def solve(self, b, x, tol=1e-10, max_it=1000, mixed=False, inner_tol=1e-4, check_every=0, inner_max_it=1000):
        p = make_params(tol=tol, max_it=max_it, mixed=mixed, inner_tol=inner_tol, check_every=check_every,
                        inner_max_it=inner_max_it)
        st = SolveStats()
        check(lib().mfx_mg_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(st), _stream()))
        return st.as_dict()


class _OpView(Operator):
    """An operator owned by something else (a multigrid level): same methods, never destroyed here."""

    def __init__(self, handle, degree, info, owner):
        self._handle = handle
        self.degree = degree
        self._info = info
        self._owner = owner  # keeps the hierarchy alive

    @property
    def handle(self):
        return self._handle

    @handle.setter
    def handle(self, v):
        pass

    def __del__(self):
        pass
