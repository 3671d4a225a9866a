"""CPU-only checks of the C ABI library: it loads, exports every function
that include/gmg.h declares, validates descriptors before touching a device,
and its host-side set-up math (the fast-diagonalisation data of App. A.3) is
right: closed forms for Q1, the generalised eigen identities, and the
tensor-product inverse against a brute-force dense inverse of the oracle's
assembled patch matrix."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.mesh import Mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gmg():
    from paper_2407_02100_gb300 import build, gmg as g
    build.build()
    return g


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    pat = r"^\s*(?:const\s+)?(?:long\s+long|\w+)\*?\s+\*?(\w+)\s*\("
    return sorted(set(re.findall(pat, src, flags=re.M)))


def test_library_exports_every_declared_function(gmg):
    names = _declared_functions()
    assert "gmg_smooth" in names and "cg_gmg_solve" in names and "gmg_vcycle" in names
    L = gmg.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(gmg.EXPORTS) == names


def test_status_strings(gmg):
    assert gmg.gmg_status_string(0) == "ok"
    assert gmg.gmg_status_string(-1) == "invalid argument"
    assert gmg.gmg_status_string(12345) == "unknown status"


@pytest.mark.parametrize("bad", [dict(dim=4), dict(degree=0), dict(degree=9), dict(n_cells=1),
                                 dict(n_levels=-1), dict(precision=7),
                                 dict(damping=float("nan")), dict(pre_sweeps=-1)])
def test_create_rejects_bad_descriptors(gmg, bad):
    """Rejected by the host-side validation, before any CUDA call."""
    args = dict(dim=2, degree=2, n_cells=8, n_levels=0, precision=0, damping=1.0,
                pre_sweeps=1, post_sweeps=1)
    args.update(bad)
    desc = gmg.GmgDesc(args["dim"], args["degree"], args["n_cells"], args["n_levels"],
                       args["precision"], args["damping"], args["pre_sweeps"], args["post_sweeps"], None)
    h = ctypes.c_void_p()
    assert gmg.lib().gmg_create(ctypes.byref(desc), ctypes.byref(h)) == -1
    assert not h.value
    assert gmg.lib().gmg_create(None, ctypes.byref(h)) == -1


def test_null_problem_is_rejected(gmg):
    L = gmg.lib()
    assert L.gmg_smooth(None, 0, None, None, 1, 0) == -1
    assert L.gmg_vcycle(None, None, None) == -1
    assert L.gmg_destroy(None) == 0
    assert L.gmg_set_shared_faces(None, 1) == -1
    assert L.gmg_shared_faces(None) == -1
    assert L.gmg_set_three_pass_operator(None, 1) == -1
    assert L.gmg_three_pass_operator(None) == -1


def test_header_is_plain_c():
    """The boundary header compiles as strict C99 (no C++ constructs)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = '#include "include/gmg.h"\nint main(void) { return 0; }\n'
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", ROOT, "-x", "c", "-"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_q1_patch_closed_form(gmg):
    """k = 1: the patch interior is the vertex; on two unit cells
    M = 2/3, K = 2, so lambda = 3 and T = sqrt(3/2)."""
    M, K, T, lam = gmg.gmg_patch_fd_1d(1)
    assert abs(M[0, 0] - 2 / 3) < 1e-15 and abs(K[0, 0] - 2) < 1e-15
    assert abs(lam[0] - 3) < 1e-14 and abs(abs(T[0, 0]) - np.sqrt(1.5)) < 1e-15


@pytest.mark.parametrize("k", range(1, 9))
def test_generalised_eigen_identities(gmg, k):
    M, K, T, lam = gmg.gmg_patch_fd_1d(k)
    m = 2 * k - 1
    assert np.abs(T.T @ M @ T - np.eye(m)).max() < 1e-13
    assert np.abs(T.T @ K @ T - np.diag(lam)).max() < 1e-12 * lam.max()
    assert np.all(lam > 0)


@pytest.mark.parametrize("dim,k", [(2, k) for k in range(1, 9)] + [(3, k) for k in range(1, 6)])
def test_fd_inverse_equals_dense_inverse(gmg, dim, k):
    """(T x T [x T]) diag(1/sum lambda) (T x T [x T])^T equals inv(A_j) of the
    oracle's patch block assembled from full-quadrature cell matrices (unit
    cells, h = 1)."""
    M, K, T, lam = gmg.gmg_patch_fd_1d(k)
    mesh = Mesh(dim, k, 2)                    # n = 2: one patch; h = 1/2
    Abar, inner = mesh.patch_block()
    Aj = Abar[:, inner] / mesh.h ** (dim - 2)  # unit cells
    S = T
    for _ in range(dim - 1):
        S = np.kron(S, T)                     # kron(T_z, T_y, T_x): x index fastest
    lsum = lam.copy()
    for _ in range(dim - 1):
        lsum = np.add.outer(lsum, lam).ravel()
    Ainv_fd = S @ np.diag(1.0 / lsum) @ S.T
    Ainv = np.linalg.inv(Aj)
    assert np.abs(Ainv_fd - Ainv).max() < 1e-12 * np.abs(Ainv).max() * max(1.0, np.linalg.cond(Aj) / 1e3)
