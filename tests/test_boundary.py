"""C-ABI boundary checks that need no GPU: the library loads, exports every function
include/absorber.h declares, its struct layouts match the binding, and its sparsity
patterns equal the oracle's structural patterns bit for bit."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import absorber_inputs as ai
from oracle import model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_2607_15420_gb300 import build
    build.build()
    from paper_2607_15420_gb300 import binding as b
    b.lib()
    return b


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "absorber.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:abs_status|void|const char\*|int64_t|int32_t)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_match_header(binding):
    names = _declared_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert n in binding.EXPORTS, f"binding lacks {n}"


def test_struct_layouts(binding):
    for i, s in enumerate(binding.STRUCTS):
        assert binding.lib().abs_struct_size(i) == ctypes.sizeof(s), s.__name__
    assert binding.lib().abs_struct_size(99) == -1


def _oracle_pattern():
    P = ai.PARAMS
    F = ai.make_feeds(1, 3)
    Z, d = model.initial_point(P, F)
    rng = np.random.default_rng(11)
    Z = np.abs(Z) * rng.uniform(0.5, 1.5, Z.shape) + 0.05
    Z.reshape(1, model.N, model.NV)[:, :, model.IT] = 3.2
    lam = rng.standard_normal(Z.shape)
    _, J, Jd, W, Wdd = model.derivatives(P, F, Z, d, lam)
    Jf = np.concatenate([J[0], Jd[0][:, None]], axis=1)        # column 220 = d
    jr, jc = np.nonzero(Jf)                                     # row-major = CSR order
    Wl = np.tril(W[0])
    hr, hc = np.nonzero(Wl)
    hr = np.append(hr, model.NS)
    hc = np.append(hc, model.NS)
    assert Wdd[0] != 0.0
    return jr, jc, hr, hc


def test_pattern_bit_exact_vs_oracle(binding):
    jr, jc, hr, hc = binding.scenario_pattern()
    ojr, ojc, ohr, ohc = _oracle_pattern()
    np.testing.assert_array_equal(jr, ojr)
    np.testing.assert_array_equal(jc, ojc)
    np.testing.assert_array_equal(hr, ohr)
    np.testing.assert_array_equal(hc, ohc)


def test_create_without_gpu_fails_loudly(binding):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.AbsorberError):
        binding.Problem(ai.PARAMS, ai.make_feeds(2, 0))
