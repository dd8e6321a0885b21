"""CPU tests of the partitioned operator's bookkeeping (the distributed path of Sec. 2.6 / Sec. 3.7).

mfx_partition_box (host-only) splits a structured box into slabs of cells along z.  Checked here:
the slabs tile the box, each part's lattice is the contiguous slice of the global vector it claims,
owned DoFs count every DoF once, interface faces are natural on the parts.  Then two gloo ranks
(world size 2, CPU) each apply the oracle's operator of their own slab (the stand-in for the part's
GPU vmult), exchange their shared plane, add the neighbour's partial values except on Dirichlet points,
and must reproduce the rows of the oracle's global operator; the same ranks run Jacobi-PCG with two
allreduces per iteration and must reach the global solution.
"""
import os
import socket

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle import mesh as omesh
from paper_1910_13247_gb300 import build as mbuild
from paper_1910_13247_gb300 import mfx, synthetic


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    mfx.lib()


@pytest.mark.parametrize("nz,n_parts", [(1, 1), (5, 2), (7, 3), (8, 8), (10, 4)])
@pytest.mark.parametrize("k", [1, 3])
def test_parts_tile_the_box_and_the_vector(nz, n_parts, k):
    nx, ny = 3, 2
    plane = (k * nx + 1) * (k * ny + 1)
    n_global = plane * (k * nz + 1)
    infos = [mfx.partition_box(nx, ny, nz, k, n_parts, p, dirichlet=0b111101) for p in range(n_parts)]
    assert infos[0].cz0 == 0 and sum(i.nz for i in infos) == nz
    assert max(i.nz for i in infos) - min(i.nz for i in infos) <= 1
    owned = 0
    for p, i in enumerate(infos):
        assert i.plane == plane and i.n_dofs == plane * (k * i.nz + 1)
        assert i.dof0 == plane * k * i.cz0 and i.vertex0 == (nx + 1) * (ny + 1) * i.cz0
        assert (i.has_lo, i.has_hi) == (int(p > 0), int(p < n_parts - 1))
        if p + 1 < n_parts:  # the upper plane of part p is the lower plane of part p + 1
            assert infos[p + 1].cz0 == i.cz0 + i.nz and infos[p + 1].dof0 == i.dof0 + i.n_dofs - plane
        # interfaces are natural on the part, the other faces keep the global mask
        assert i.dirichlet & 0b001111 == 0b001101
        assert bool(i.dirichlet & 16) == (p == 0) and bool(i.dirichlet & 32) == (p == n_parts - 1)
        assert i.n_owned == i.n_dofs - (plane if i.has_hi else 0)
        owned += i.n_owned
    assert owned == n_global


def test_partition_errors():
    for args in [(3, 2, 4, 2, 5, 0), (3, 2, 4, 2, 2, 2), (3, 2, 4, 2, 0, 0), (0, 2, 4, 2, 1, 0)]:
        with pytest.raises(mfx.MfxError) as e:
            mfx.partition_box(*args)
        assert e.value.code == mfx.EINVAL
    with pytest.raises(mfx.MfxError) as e:
        mfx.partition_box(3, 2, 4, 9, 2, 0)
    assert e.value.code == mfx.EUNSUPPORTED


def slab_operator(nx, ny, nz, k, verts, info):
    """The oracle's operator of one part's slab (interface faces natural), and its slice of the vertex lattice."""
    nv = (nx + 1) * (ny + 1) * (info.nz + 1)
    v = verts[info.vertex0:info.vertex0 + nv]
    om = omesh.structured_mesh(nx, ny, info.nz, k, v, dirichlet=info.dirichlet)
    return fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))


def free_mask_of_plane(nx, ny, k, dirichlet):
    Mx, My = k * nx + 1, k * ny + 1
    I, J = np.meshgrid(np.arange(Mx), np.arange(My), indexing="xy")
    d = np.zeros(I.shape, dtype=bool)
    if dirichlet & 1:
        d |= I == 0
    if dirichlet & 2:
        d |= I == Mx - 1
    if dirichlet & 4:
        d |= J == 0
    if dirichlet & 8:
        d |= J == My - 1
    return ~d.reshape(-1)


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mfx.lib()
        nx, ny, nz, k, mask = 3, 2, 5, 2, 0b111111
        verts = synthetic.deformed_vertices(nx, ny, nz)
        info = mfx.partition_box(nx, ny, nz, k, world, rank, dirichlet=mask)
        K_loc = slab_operator(nx, ny, nz, k, verts, info)
        om = omesh.structured_mesh(nx, ny, nz, k, verts, dirichlet=mask)
        K = fem.assemble(om, k + 1, fem.COEF_TRIG, (1.0, 0.5))
        sl = slice(info.dof0, info.dof0 + info.n_dofs)
        free = free_mask_of_plane(nx, ny, k, info.dirichlet)
        P = info.plane

        def exchange_sum(v):
            """Send the partial shared planes, add the neighbour's on the free points."""
            reqs, bufs = [], {}
            if info.has_lo:
                bufs[0] = torch.empty(P, dtype=torch.float64)
                reqs += [dist.isend(torch.tensor(v[:P]), rank - 1), dist.irecv(bufs[0], rank - 1)]
            if info.has_hi:
                bufs[1] = torch.empty(P, dtype=torch.float64)
                reqs += [dist.isend(torch.tensor(v[-P:]), rank + 1), dist.irecv(bufs[1], rank + 1)]
            for r in reqs:
                r.wait()
            v = v.copy()
            if 0 in bufs:
                v[:P][free] += bufs[0].numpy()[free]
            if 1 in bufs:
                v[-P:][free] += bufs[1].numpy()[free]
            return v

        def allreduce(vals):
            t = torch.tensor(vals, dtype=torch.float64)
            dist.all_reduce(t)
            return t.numpy()

        # vmult: local product, exchange; equals the global rows of this part's slice
        x = synthetic.uniform_vector(om.n_dofs, 7)
        y = exchange_sum(K_loc @ x[sl])
        ref = (K @ x)[sl]
        err = np.abs(y - ref).max() / np.abs(K @ x).max()
        # Jacobi-PCG with two allreduces per iteration over owned DoFs
        b = synthetic.gaussian_vector(om.n_dofs, 8)
        b[om.constrained] = 0.0
        bl = b[sl]
        own = slice(0, info.n_owned)
        D = exchange_sum(K_loc.diagonal())
        xl = np.zeros_like(bl)
        r = bl.copy()
        z = r / D
        p = z.copy()
        bb, rz = allreduce([bl[own] @ bl[own], r[own] @ z[own]])
        rr, it, n_allreduce = bb, 0, 1
        while rr > 1e-20 * bb:
            q = exchange_sum(K_loc @ p)
            pq = allreduce([p[own] @ q[own]])[0]
            alpha = rz / pq
            xl += alpha * p
            r -= alpha * q
            z = r / D
            rz_new, rr = allreduce([r[own] @ z[own], r[own] @ r[own]])
            n_allreduce += 2
            p = z + (rz_new / rz) * p
            rz = rz_new
            it += 1
        xd = spla.spsolve(K.tocsc(), b)[sl]
        sol_err = np.linalg.norm(xl - xd) / np.linalg.norm(spla.spsolve(K.tocsc(), b))
        out.put((rank, float(err), float(sol_err), it, n_allreduce))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_global_operator_and_solve():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, err, sol_err, it, n_allreduce in res:
        assert err < 1e-13, (rank, err)
        assert sol_err < 1e-8, (rank, sol_err)
        assert n_allreduce == 2 * it + 1
    assert res[0][3] == res[1][3]  # both ranks took the same iterations
