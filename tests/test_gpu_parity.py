"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle on the same seeded inputs, element by element.

Tolerance (FP64): relative 1e-12 in the 2-norm and 1e-11 of the largest
entry elementwise.  The fast-diagonalisation local solve and the oracle's
LU solve round differently; their gap grows with the condition number of
A_j, which stays below ~1e4 for k <= 8, i.e. ~1e-12 relative.
Sizes span several operator tiles and ragged tails (n not a multiple of the
tile edge), Q1..Q8, 2D and 3D, boundary patches included."""
import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.multigrid import Multigrid, prolongation
from oracle.smoother import PatchSmoother
from paper_2407_02100_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def gmg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


def close(got, ref, rtol=RTOL, what=""):
    scale = np.abs(ref).max()
    err2 = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    errm = np.abs(got - ref).max() / max(scale, 1e-300)
    assert err2 <= rtol and errm <= 10 * rtol, f"{what}: rel2={err2:.3e} relmax={errm:.3e}"


OPERATOR_CASES = [(2, 1, 37), (2, 2, 20), (2, 3, 9), (2, 5, 7), (2, 8, 5),
                  (3, 1, 10), (3, 2, 10), (3, 3, 5), (3, 4, 5), (3, 5, 3), (3, 7, 3)]


@pytest.mark.parametrize("dim,k,n", OPERATOR_CASES)
def test_apply_operator(gmg, dim, k, n):
    m = Mesh(dim, k, n)
    P = gmg.Problem(dim, k, n, n_levels=1)
    x = inputs.random_nodal(dim, k, n, 101)
    y = P.zeros()
    gmg.gmg_apply_operator(P.h, 0, P.to_device(x), y)
    close(P.from_device(y), m.assemble() @ x, what="A x")


SWEEP_CASES = [(2, 1, 9), (2, 2, 32), (2, 3, 11), (2, 4, 6), (2, 6, 5), (2, 8, 4),
               (3, 1, 9), (3, 2, 7), (3, 3, 6), (3, 4, 5), (3, 5, 4), (3, 6, 3), (3, 8, 3)]


# FP64 colour steps of up to max_patches patches run on the coarse-level kernel
# (one output per thread); small=1024 takes it for every colour of these
# meshes, small=0 the closure / shared-face kernels
@pytest.mark.parametrize("dim,k,n", SWEEP_CASES)
@pytest.mark.parametrize("small", [1024, 0])
def test_each_colour_step(gmg, dim, k, n, small):
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(dim, k, n, n_levels=1, small_sweep=small)
    u0 = inputs.random_nodal(dim, k, n, 201)
    b = inputs.random_nodal(dim, k, n, 202)
    bd = P.to_device(b)
    for c in range(m.n_colours):
        ud = P.to_device(u0)
        gmg.gmg_smooth_colour(P.h, 0, ud, bd, c)
        ref = s.colour_step(u0.copy(), b, c)
        close(P.from_device(ud), ref, what=f"colour {c}")


@pytest.mark.parametrize("dim,k,n", SWEEP_CASES)
@pytest.mark.parametrize("reverse", [False, True])
@pytest.mark.parametrize("small", [1024, 0])
def test_full_sweep(gmg, dim, k, n, reverse, small):
    m = Mesh(dim, k, n)
    s = PatchSmoother(m)
    P = gmg.Problem(dim, k, n, n_levels=1, small_sweep=small)
    u0 = inputs.random_nodal(dim, k, n, 301)
    b = inputs.random_nodal(dim, k, n, 302)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 2, reverse)
    ref = s.sweep(s.sweep(u0, b, reverse), b, reverse)
    close(P.from_device(ud), ref, what="two sweeps")


@pytest.mark.parametrize("omega", [0.7, 1.3])
@pytest.mark.parametrize("small", [1024, 0])
def test_damped_sweep(gmg, omega, small):
    dim, k, n = 3, 2, 6
    m = Mesh(dim, k, n)
    s = PatchSmoother(m, omega)
    P = gmg.Problem(dim, k, n, n_levels=1, damping=omega, small_sweep=small)
    u0 = inputs.random_nodal(dim, k, n, 401)
    b = inputs.random_nodal(dim, k, n, 402)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 1, False)
    close(P.from_device(ud), s.sweep(u0, b), what="damped sweep")


# FP64 problems run the transfers in double-float arithmetic (one coarse
# cell of outputs per thread): the cases span several coarse cells per axis,
# degrees up to 8 and both dimensions
TRANSFER_CASES = [(2, 1, 8), (2, 2, 6), (2, 3, 4), (2, 5, 4), (2, 8, 4), (3, 1, 6), (3, 2, 4), (3, 3, 4),
                  (3, 3, 6), (3, 4, 2), (3, 4, 4), (3, 7, 2), (3, 8, 2)]


@pytest.mark.parametrize("dim,k,n", TRANSFER_CASES)
def test_restrict_and_prolongate(gmg, dim, k, n):
    c, f = Mesh(dim, k, n // 2), Mesh(dim, k, n)
    Pm = prolongation(c, f)
    P = gmg.Problem(dim, k, n, n_levels=2)
    rf = inputs.random_nodal(dim, k, n, 501)
    ec = inputs.random_nodal(dim, k, n // 2, 502)
    uf = inputs.random_nodal(dim, k, n, 503)
    out_c = P.zeros(0)
    gmg.gmg_restrict(P.h, 1, P.to_device(rf, 1), out_c)
    close(P.from_device(out_c, 0), Pm.T @ rf, what="restrict")
    ufd = P.to_device(uf, 1)
    gmg.gmg_prolongate_add(P.h, 0, P.to_device(ec, 0), ufd)
    close(P.from_device(ufd, 1), uf + Pm @ ec, what="prolongate")


@pytest.mark.parametrize("dim,k,n", [(2, 2, 4), (2, 4, 3), (2, 8, 2), (3, 1, 4), (3, 2, 3), (3, 4, 2), (3, 7, 2)])
def test_coarse_solve(gmg, dim, k, n):
    m = Mesh(dim, k, n)
    A = m.assemble()
    P = gmg.Problem(dim, k, n, n_levels=1)
    b = inputs.random_nodal(dim, k, n, 601)
    x = P.zeros(0)
    gmg.gmg_coarse_solve(P.h, P.to_device(b, 0), x)
    xg = P.from_device(x, 0)
    inner = m.interior_nodes()
    ref = np.zeros_like(b)
    ref[inner] = np.linalg.solve(A[inner][:, inner].toarray(), b[inner])
    close(xg, ref, what="coarse solve")


VCYCLE_CASES = [(2, 2, 32, 3), (2, 3, 16, 3), (2, 1, 16, 4), (3, 2, 8, 3), (3, 3, 4, 2), (3, 4, 4, 2)]


@pytest.mark.parametrize("dim,k,n,L", VCYCLE_CASES)
def test_vcycle(gmg, dim, k, n, L):
    mg = Multigrid(dim, k, n, L)
    P = gmg.Problem(dim, k, n, n_levels=L)
    b = inputs.random_nodal(dim, k, n, 701)
    x = P.zeros()
    gmg.gmg_vcycle(P.h, x, P.to_device(b))
    close(P.from_device(x), mg.vcycle(b), what="V-cycle")


@pytest.mark.parametrize("dim,k,n,L", VCYCLE_CASES)
def test_pcg(gmg, dim, k, n, L):
    mg = Multigrid(dim, k, n, L)
    P = gmg.Problem(dim, k, n, n_levels=L)
    b = inputs.random_nodal(dim, k, n, 801)
    u = P.zeros(dtype=__import__("torch").float64)
    status, st = gmg.cg_gmg_solve(P.h, u, P.to_device(b, dtype=__import__("torch").float64), 1e-10, 100)
    xo, its, hist = mg.pcg(b, rtol=1e-10)
    assert st.converged == 1 and st.relative_residual <= 1e-10
    assert abs(st.iterations - its) <= 1, (st.iterations, its)
    got = P.from_device(u)
    assert np.linalg.norm(got - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("dim,k,n,prec", [(3, 4, 5, 0), (3, 3, 6, 1), (2, 3, 9, 1), (3, 2, 7, 0)])
def test_tma_and_elementwise_gathers_agree(gmg, dim, k, n, prec):
    """Vectors whose base is not 16-byte aligned cannot be read by TMA boxes:
    the sweep then gathers element by element.  Both gathers feed the same
    arithmetic, so the results must be bit-identical, and equal to the
    oracle's sweep to the precision's bound."""
    import torch
    P = gmg.Problem(dim, k, n, n_levels=1, precision=prec, small_sweep=0)
    u0 = inputs.random_nodal(dim, k, n, 5001)
    b = inputs.random_nodal(dim, k, n, 5002)
    ua = P.to_device(u0)
    bd = P.to_device(b)
    gmg.gmg_smooth(P.h, 0, ua, bd, 1, False)
    buf = torch.zeros(ua.numel() + 1, dtype=ua.dtype, device=ua.device)
    um = buf[1:]                                  # 4 or 8 bytes off 16-byte alignment
    um.copy_(P.to_device(u0))
    gmg.gmg_smooth(P.h, 0, um, bd, 1, False)
    assert gmg.gmg_tc_status() == 0
    assert torch.equal(ua, um)
    ref = PatchSmoother(Mesh(dim, k, n)).sweep(u0, b)
    got = P.from_device(ua)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < (1e-12 if prec == 0 else 1e-5)


# degenerate meshes: one interior vertex per direction, so a single patch in
# the last colour and empty launches for every other colour
@pytest.mark.parametrize("dim,k,n", [(2, 3, 2), (3, 2, 2), (3, 4, 2)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("small", [1024, 0])
def test_single_patch_mesh(gmg, dim, k, n, prec, small):
    m = Mesh(dim, k, n)
    P = gmg.Problem(dim, k, n, n_levels=1, precision=prec, small_sweep=small)
    u0 = inputs.random_nodal(dim, k, n, 5201)
    b = inputs.random_nodal(dim, k, n, 5202)
    ud = P.to_device(u0)
    gmg.gmg_smooth(P.h, 0, ud, P.to_device(b), 1, False)
    close(P.from_device(ud), PatchSmoother(m).sweep(u0, b), 1e-12 if prec == 0 else 1e-5, "single patch")


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_full_size_colour_step_on_sampled_patches(gmg, prec, tol):
    """3D Q4 on 64^3 cells (16,974,593 nodes), the bench's workload and launch
    configuration: one colour step on the GPU, then 40 sampled patches of
    that colour recomputed one by one by the oracle (dense local solve of the
    patch block built from the same inputs).  Nodes outside the colour's
    patch interiors must be untouched."""
    dim, k, n, colour = 3, 4, 64, 5
    m = Mesh(dim, k, n)
    P = gmg.Problem(dim, k, n, n_levels=1, precision=prec)
    u0 = inputs.random_nodal(dim, k, n, 5301)
    b = inputs.random_nodal(dim, k, n, 5302)
    if prec == 1:   # the FP32 kernel sees these values: the oracle takes the same
        u0 = u0.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    ud = P.to_device(u0)
    gmg.gmg_smooth_colour(P.h, 0, ud, P.to_device(b), colour)
    got = P.from_device(ud)
    V = m.vertices_of_colour(colour)
    rng = np.random.default_rng(5303)
    sample = V[rng.choice(len(V), 40, replace=False)]
    Abar, inner = m.patch_block()
    Aj = Abar[:, inner]
    clo, inn = m.closure_index(sample), m.interior_index(sample)
    r = b[inn] - u0[clo] @ Abar.T
    ref = u0[inn] + np.linalg.solve(Aj, r.T).T
    close(got[inn].ravel(), ref.ravel(), tol, "sampled patches")
    touched = np.zeros(m.n_nodes, dtype=bool)
    touched[m.interior_index(V).ravel()] = True
    assert np.array_equal(got[~touched], u0[~touched])


@pytest.mark.parametrize("dim,k,ns,prec", [(2, 2, (8, 16, 32), 0), (2, 3, (4, 8, 16), 1),
                                           (3, 2, (4, 8, 16), 0), (3, 4, (2, 4, 8), 1)])
def test_manufactured_solution_solved_on_the_gpu_converges(gmg, dim, k, ns, prec):
    """-Laplace u = f with u = prod sin(pi x_a) (App. A.2's test problem):
    the GPU GMG-PCG solution (FP64, or FP32 V-cycle in FP64 CG) of the
    discrete problem has an L2 error falling at O(h^(k+1)) and matches the
    oracle's direct solution of the same system."""
    import torch
    from oracle import problem
    u_exact, f = problem.sine_solution(dim)
    errs = []
    for n in ns:
        m = Mesh(dim, k, n)
        b = problem.load_vector(m, f)
        P = gmg.Problem(dim, k, n, precision=prec)
        u = P.zeros(dtype=torch.float64)
        _, st = gmg.cg_gmg_solve(P.h, u, P.to_device(b, dtype=torch.float64), 1e-12, 100)
        assert st.converged
        got = P.from_device(u)
        errs.append(problem.l2_error(m, got, u_exact))
        if n == ns[0]:
            A = m.assemble()
            inner = m.interior_nodes()
            ref = np.zeros_like(b)
            import scipy.sparse.linalg as spla
            ref[inner] = spla.spsolve(A[inner][:, inner].tocsc(), b[inner])
            close(got, ref, 1e-10, "direct solution")
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > k + 1 - 0.3, (errs, rates)
