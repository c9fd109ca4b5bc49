"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every function include/a2ls.h declares, rejects bad arguments before touching
a device, and its small dense eigensolver (host-compiled) agrees with LAPACK."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
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


@pytest.mark.parametrize("kind", ["random", "scaled", "clustered", "near_identity"])
def test_small_eigensolver_matches_lapack(small_eig_exe, kind):
    rng = np.random.Generator(np.random.PCG64(hash(kind) % 1000))
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
