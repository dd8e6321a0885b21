"""Usage example of the library from Python (device vectors are torch tensors; the library
allocates none of them): FP64 and FP32 vmult, a mixed-precision Chebyshev-Jacobi PCG solve, the
geometric multigrid solve and one request to the solve server.

    python -m paper_1910_13247_gb300.example        (needs a GPU and the built library)
"""
import time

import torch

from paper_1910_13247_gb300 import mfx, synthetic

n, k = 24, 4
mesh = mfx.Mesh.structured_box(n, n, n, synthetic.deformed_vertices(n, n, n))  # Dirichlet on every face
op = mfx.Operator(mesh, k, mfx.COEF_TRIG, (1.0, 0.5))  # a(x) = 1 + 0.5 sin(2 pi x) cos(2 pi y) z

x = torch.rand(op.n_dofs, dtype=torch.float64, device="cuda")
y = torch.empty_like(x)
op.vmult(x, y)                                   # FP64 vmult
x32, y32 = x.float(), torch.empty(op.n_dofs, dtype=torch.float32, device="cuda")
op.vmult(x32, y32)                               # FP32 vmult (float32 tensors select it)

b = torch.ones(op.n_dofs, dtype=torch.float64, device="cuda")
op.distribute(b)                                 # constrained rows of b as the constraints give them
u = torch.zeros_like(b)
st = op.solve(b, u, tol=1e-10, precond=mfx.PRECOND_CHEBYSHEV, mixed=True)  # FP32 PCG in FP64 correction
assert st["status"] == 0

mg = mfx.Multigrid(mesh, k, mfx.COEF_TRIG, (1.0, 0.5))  # geometric multigrid hierarchy
um = torch.zeros_like(b)
assert mg.solve(b, um, tol=1e-10, mixed=True)["status"] == 0

srv = mfx.Server(budget_bytes=8 << 30)           # continuous-batching solve server
leaves = synthetic.octree_leaves(4, 2, (0.5, 0.5, 0.5), 0.3)  # 4^3 coarse cells refined twice in a ball
t = srv.submit(3, leaves=leaves, n_coarse=4)     # Q3 on the octree, b = 1, mixed precision
while srv.poll(t)["state"] < mfx.REQ_DONE:
    time.sleep(1e-3)
assert srv.poll(t)["state"] == mfx.REQ_DONE
u_octree = srv.result(t)                         # host copy of the solution
srv.retire(t)
srv.close()
print("example ok:", op.n_dofs, "DoFs;", "octree solution of", u_octree.size, "DoFs")
