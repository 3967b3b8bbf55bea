"""The partitioned operator of the multi-GPU decomposition (A = sum_k P_k^T A_k P_k, Sec. 2.3),
emulated on one GPU: the mesh is cut into z-slabs, each slab is an operator of its own on its
sub-mesh and its own node grid, P_k restricts the global vector to the slab's nodes, and the
interface planes shared by neighbouring slabs are summed (the halo exchange).  The result must
equal the monolithic action (relative l2 <= 1e-12): the one-exchange-per-action structure the
replicas-only benchmark does not exercise."""
import numpy as np
import pytest

import fem_inputs as FI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def F():
    import paper_2402_15940_b300 as mod
    return mod


def slabs(nz, k):
    cuts = np.linspace(0, nz, k + 1).round().astype(int)
    return [(int(cuts[i]), int(cuts[i + 1])) for i in range(k)]


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p,shape,k", [(2, (3, 4, 6), 3), (4, (2, 3, 5), 2), (3, (3, 2, 7), 4)])
def test_slab_partitioned_action_equals_monolithic(p, shape, k, form):
    nx, ny, nz = shape
    verts = FI.perturbed_cube_vertices(nx, ny, nz, seed=p)
    whole = F().Operator(nx, ny, nz, verts, p, form=form)
    Nx, Ny = p * nx + 1, p * ny + 1
    plane = Nx * Ny                               # nodes per z-plane of the global node grid
    vplane = (nx + 1) * (ny + 1)                  # vertices per z-plane
    x = torch.from_numpy(FI.uniform_vector(whole.N, seed=3)).cuda()
    y_ref = whole.apply(x)
    y = torch.zeros_like(x)
    for z0, z1 in slabs(nz, k):
        part = F().Operator(nx, ny, z1 - z0, verts[z0 * vplane:(z1 + 1) * vplane], p, form=form)
        lo, hi = z0 * p * plane, (z1 * p + 1) * plane     # the slab's node planes, interfaces included
        assert part.N == hi - lo
        y[lo:hi] += part.apply(x[lo:hi].contiguous())     # P_k^T A_k P_k x; shared planes summed
    err = float((y - y_ref).norm() / y_ref.norm())
    assert err <= 1e-12, err
