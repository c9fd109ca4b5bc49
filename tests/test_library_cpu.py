"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every function include/a2ls.h declares, rejects bad arguments before touching
a device, links into a strict C99 program, and its small dense eigensolver
(host-compiled) agrees with LAPACK."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import scipy.linalg as sla
import pytest

from paper_2201_02250_gb300 import a2ls, _build

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return a2ls.lib(build_if_missing=False)


def test_exports_every_declared_symbol(lib):
    names = a2ls.header_functions()
    assert {"a2ls_setup", "a2ls_apply", "a2ls_solve", "a2ls_destroy"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = a2ls.default_options()
    assert (o.precision, o.variant, o.pou, o.restart, o.max_it, o.flexible) == (0, 0, 0, 30, 1000, -1)
    assert (o.eig_block_size, o.static_pivoting) == (0, 0)


def test_argument_errors_without_device(lib):
    h = ctypes.c_void_p()
    rc = lib.a2ls_setup(None, None, 1, 4, None, ctypes.byref(h))
    assert rc == a2ls.A2LS_ERR_ARG and not h.value
    assert b"null" in lib.a2ls_last_error()
    csr = a2ls.CSR(0, 0, None, None, None)
    rc = lib.a2ls_setup(ctypes.byref(csr), ctypes.c_void_p(8), 1, 4, None, ctypes.byref(h))
    assert rc == a2ls.A2LS_ERR_ARG and b"positive" in lib.a2ls_last_error()
    assert lib.a2ls_apply(None, None, None) == a2ls.A2LS_ERR_ARG
    assert lib.a2ls_query(None, 0, None, 0, None) == a2ls.A2LS_ERR_ARG
    lib.a2ls_destroy(None)
    assert lib.a2ls_trim_memory() == 0  # no pool exists before the first setup on a device


@pytest.mark.parametrize("field,value,words", [
    ("precision", 9, b"precision"), ("variant", 17, b"variant"), ("pou", 5, b"partition of unity"),
    ("static_pivoting", 2, b"static_pivoting"), ("local_solve_kernel", 7, b"local_solve_kernel"),
])
def test_option_errors_without_device(lib, field, value, words):
    # options are checked before the CSR arrays are touched: placeholder pointers are never read
    csr = a2ls.CSR(4, 4, 8, 8, 8)
    o = a2ls.default_options(**{field: value})
    h = ctypes.c_void_p()
    rc = lib.a2ls_setup(ctypes.byref(csr), ctypes.c_void_p(8), 1, 2, ctypes.byref(o), ctypes.byref(h))
    assert rc == a2ls.A2LS_ERR_ARG and not h.value
    assert words in lib.a2ls_last_error()


def test_streaming_local_solves_refused_for_fp64_without_device(lib):
    csr = a2ls.CSR(4, 4, 8, 8, 8)
    o = a2ls.default_options(precision="fp64", local_solve_kernel=3000)
    h = ctypes.c_void_p()
    rc = lib.a2ls_setup(ctypes.byref(csr), ctypes.c_void_p(8), 1, 2, ctypes.byref(o), ctypes.byref(h))
    assert rc == a2ls.A2LS_ERR_ARG and b"FP32 or BF16" in lib.a2ls_last_error()


def test_c_program_compiles_links_and_calls_the_abi(lib, tmp_path):
    # include/a2ls.h as strict C99 (no C++ in the header), C linkage of the exported symbols, and the
    # entry points that need no GPU: default options, a2ls_partition, argument errors
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "c_consumer")
    libdir = os.path.dirname(_build.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(os.path.dirname(HERE), "include"), os.path.join(HERE, "cpp", "c_consumer.c"),
                    "-L", libdir, "-lA2LS", "-Wl,-rpath," + libdir, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAILED" not in r.stdout and r.stdout.count("ok:") >= 10


@pytest.fixture(scope="module")
def small_eig_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("se") / "small_eig_host")
    subprocess.run([gxx, "-O2", "-x", "c++", os.path.join(HERE, "cpp", "small_eig_host.cpp"), "-o", exe, "-lm"],
                   check=True)
    return exe


def _run_small_eig(exe, H):
    m = H.shape[0]
    inp = f"{m}\n" + "\n".join(" ".join(f"{v:.17g}" for v in row) for row in H)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rc = int(out[0])
    ev = np.array([[float(t) for t in line.split()] for line in out[1:1 + m]])
    res = [float(line.split()[1]) for line in out[1 + m:] if line.startswith("res")]
    return rc, ev[:, 0] + 1j * ev[:, 1], res


KINDS = ["random", "scaled", "clustered", "near_identity"]


@pytest.mark.parametrize("kind", KINDS)
def test_small_eigensolver_matches_lapack(small_eig_exe, kind):
    rng = np.random.Generator(np.random.PCG64(101 + KINDS.index(kind)))
    for trial in range(12):
        m = int(rng.integers(2, 97))
        H = rng.standard_normal((m, m))
        if kind == "scaled":
            H = H @ np.diag(np.exp(rng.uniform(-8, 8, m)))
        elif kind == "clustered":
            H = np.diag(np.repeat(rng.standard_normal(m // 3 + 1), 3)[:m]) + 1e-10 * H
        elif kind == "near_identity":
            H = np.eye(m) + 1e-9 * H
        rc, ev, res = _run_small_eig(small_eig_exe, H)
        ref = np.linalg.eigvals(H)
        scale = max(1.0, np.abs(ref).max())
        assert rc == 0
        # modulus order, conjugate pairs adjacent with +imag first
        assert np.all(np.diff(np.abs(ev)) <= 1e-12 * scale)
        # same multiset of eigenvalues
        assert np.abs(np.sort_complex(ev) - np.sort_complex(ref)).max() <= 1e-8 * scale
        # eigenvectors of tight clusters are ill-conditioned; their residuals are looser
        assert max(res) <= (1e-10 if kind in ("random", "scaled") else 1e-7) * scale


@pytest.mark.parametrize("peclet,b,s", [(50.0, 12, 3), (400.0, 12, 3), (400.0, 24, 3), (800.0, 16, 5)])
def test_small_eigensolver_on_krylov_matrices_of_a_nonnormal_operator(small_eig_exe, peclet, b, s):
    """The Rayleigh-Ritz input of the local eigensolves: the block Hessenberg projection of a
    far-from-normal operator (here the inverse of an upwind convection-diffusion matrix) onto s
    block-Krylov steps of width b, whose Ritz values come mostly in complex pairs.  Each of LAPACK's
    eigenvalues is matched within 1e-13 of its condition number times max |S|, and the leading
    eigenvectors have residuals at rounding level."""
    from workloads import pde
    A = pde.conv_diff_2d(20, peclet, np.pi / 5).toarray()
    Tm = np.linalg.inv(A)
    n = A.shape[0]
    rng = np.random.Generator(np.random.PCG64(3))
    V = np.zeros((n, (s + 1) * b))
    H = np.zeros(((s + 1) * b, s * b))
    V[:, :b], _ = np.linalg.qr(rng.standard_normal((n, b)))
    for j in range(s):
        W = Tm @ V[:, j * b:(j + 1) * b]
        jb = (j + 1) * b
        for _ in range(2):
            G = V[:, :jb].T @ W
            H[:jb, j * b:(j + 1) * b] += G
            W = W - V[:, :jb] @ G
        Q, R = np.linalg.qr(W)
        H[jb:jb + b, j * b:(j + 1) * b] = R
        V[:, jb:jb + b] = Q
    S = H[:s * b, :s * b]
    rc, ev, res = _run_small_eig(small_eig_exe, S)
    assert rc == 0
    lam, yl, xr = sla.eig(S, left=True, right=True)
    kappa = np.array([np.linalg.norm(yl[:, j]) * np.linalg.norm(xr[:, j]) / abs(yl[:, j].conj() @ xr[:, j])
                      for j in range(len(lam))])
    sn = np.abs(S).max()
    assert np.sum(np.abs(lam.imag) > 0) >= len(lam) // 2
    for l, k in zip(lam, kappa):
        assert np.min(np.abs(ev - l)) <= 1e-13 * k * sn
    assert max(res) <= 1e-12 * sn
