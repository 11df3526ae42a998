"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every symbol include/vbgs.h declares, and rejects bad arguments
before touching the device."""
from __future__ import annotations

import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def L():
    from paper_2603_08499_gb300 import build
    build.build()
    from paper_2603_08499_gb300 import vbgs
    return vbgs


def declared_symbols() -> set[str]:
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(vbgs_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(L):
    decl = declared_symbols()
    assert {"vbgs_init", "vbgs_update", "vbgs_elbo", "vbgs_get_posterior"} <= decl
    lib = C.CDLL(str(L.LIB_PATH))
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(L.EXPORTS) == decl


def test_library_is_built_for_sm103a_only(L):
    """The build compiles every CUDA source for sm_103a alone (one -gencode,
    no PTX for other targets) and the library it wrote exists."""
    from paper_2603_08499_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("gencode" in f or f.startswith("-arch") for f in B.NVCC_FLAGS)
    assert L.LIB_PATH.exists()


def _prior(K=4):
    rng = np.random.default_rng(0)
    return {"alpha0": 1.0, "beta0": 1.0, "nu0": 8.0, "m0": rng.uniform(-1, 1, (K, 6)), "W0": np.eye(6) * 100}


def test_init_rejects_bad_arguments_on_host(L):
    pr = _prior()
    lib = L.lib()
    m0 = np.ascontiguousarray(pr["m0"])
    W0 = np.ascontiguousarray(pr["W0"])

    def init(K=4, D=6, a=1.0, b=1.0, nu=8.0, W=W0, m=m0):
        p = L.vbgs_prior(a, b, nu, m.ctypes.data_as(L._DP), W.ctypes.data_as(L._DP))
        ctx = C.c_void_p()
        return lib.vbgs_init(C.byref(ctx), C.byref(p), K, D, None), ctx

    assert init(D=5)[0] == L.VBGS_EINVAL
    assert "D must be 6" in L.vbgs_last_error(None)
    assert init(K=0)[0] == L.VBGS_EINVAL
    assert init(a=0.0)[0] == L.VBGS_EINVAL
    assert init(b=-1.0)[0] == L.VBGS_EINVAL
    assert init(nu=4.0)[0] == L.VBGS_EINVAL
    assert init(W=np.ascontiguousarray(-W0))[0] == L.VBGS_EINVAL
    assert "positive definite" in L.vbgs_last_error(None)
    Wasym = W0.copy()
    Wasym[0, 1] = 1.0
    assert init(W=np.ascontiguousarray(Wasym))[0] == L.VBGS_EINVAL
    mbad = m0.copy()
    mbad[2, 3] = np.nan
    assert init(m=mbad)[0] == L.VBGS_EINVAL
    assert lib.vbgs_init(None, None, 4, 6, None) == L.VBGS_EINVAL


def test_null_context_calls_fail_cleanly(L):
    lib = L.lib()
    assert lib.vbgs_update(None, None, 0, 1, None) == L.VBGS_EINVAL
    assert lib.vbgs_elbo(None, None, 0, None, None) == L.VBGS_EINVAL
    assert lib.vbgs_get_stats(None, None) == L.VBGS_EINVAL
    assert lib.vbgs_reassign(None, None, 0, 0, 1.0, None, None, None, None) == L.VBGS_EINVAL
    lib.vbgs_destroy(None)
    assert lib.vbgs_profile_name(2) == b"pass2"


def test_valid_init_without_gpu_reports_cuda_error(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(L.VbgsError) as e:
        L.Model(_prior())
    assert e.value.code in (L.VBGS_ECUDA, L.VBGS_ENOMEM)


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point of include/vbgs.h is documented by the comment block
    above it (shared by consecutive declarations), which names the passage
    of the paper that defines the operation (Alg., Eq., Sec., Fig.) or states
    that it has no paper counterpart."""
    import re
    src = (Path(__file__).resolve().parent.parent / "include" / "vbgs.h").read_text()
    decl = re.finditer(r"^(?:int|int64_t|void|const char \*)\s*\*?\s*(vbgs_\w+)\s*\(", src, re.M)
    missing = []
    for m in decl:
        head = src[:m.start()]
        end = head.rfind("*/")
        comment = head[head.rfind("/*", 0, end):end]
        if not re.search(r"Alg\. ?\d|Eq\. ?\d|Sec\. ?\d|Fig\. ?\d|[Nn]o paper counterpart|paper has no counterpart",
                         comment):
            missing.append(m.group(1))
    assert not missing, missing


def test_reassign_binding_checks_sizes_before_the_library(L):
    """The binding rejects a Gumbel array whose length is not the point count
    before it reaches the library (no context or GPU needed)."""
    with pytest.raises(ValueError):
        L.vbgs_reassign(None, np.zeros((5, 6)), 2, np.zeros(4))
    assert L.VBGS_FLAG_SPLIT == 8
