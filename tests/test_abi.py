"""CPU checks of the C ABI: the library loads, exports every entry point that
include/cudahm.h declares, agrees with the binding on struct layouts, and rejects
bad configurations before touching a device."""
import os
import re

import pytest

from paper_2105_08026_gb300 import build as cbuild
from paper_2105_08026_gb300 import cudahm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not cbuild.up_to_date():
        try:
            cbuild.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    return cudahm.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cudahm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cudahm_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(cudahm.EXPORTED) == names


def test_struct_layouts(lib):
    import ctypes
    assert lib.cudahm_sizeof_config() == ctypes.sizeof(cudahm.CudahmConfig)
    assert lib.cudahm_sizeof_stats() == ctypes.sizeof(cudahm.CudahmStats)


def test_config_defaults(lib):
    cfg = cudahm.cudahm_config_init(cudahm.LF, 300000)
    assert cfg.abi_version == cudahm.ABI_VERSION
    assert cfg.d == 1 and cfg.n == 300000
    assert cfg.target_accept == 0.4 and abs(cfg.adapt_exponent - 2 / 3) < 1e-15
    assert cfg.model_consts[3] == 1024 and cfg.model_consts[4] == 1024
    assert cfg.debug_skip_barrier_cta == -1


@pytest.mark.parametrize("mutate,code", [
    (lambda c: setattr(c, "abi_version", 99), cudahm.EINVAL),
    (lambda c: setattr(c, "model", 7), cudahm.EINVAL),
    (lambda c: setattr(c, "d", 3), cudahm.EINVAL),
    (lambda c: setattr(c, "n", 0), cudahm.EINVAL),
    (lambda c: setattr(c, "target_accept", 1.5), cudahm.EINVAL),
    (lambda c: setattr(c, "adapt_exponent", 0.3), cudahm.EINVAL),
    (lambda c: setattr(c, "precision", 7), cudahm.EINVAL),
    (lambda c: setattr(c, "model", cudahm.MVN3), cudahm.EINVAL),  # d = 1 does not match MVN3
    (lambda c: setattr(c, "model", cudahm.BB1), cudahm.EINVAL),   # BB1 needs sigma0, alpha, nu, r_max
    (lambda c: [setattr(c, "model", cudahm.BB1), setattr(c, "precision", cudahm.FP32)] and None,
     cudahm.EUNSUPPORTED),  # BB1 has the FP64 form only
    (lambda c: c.theta_init.__setitem__(1, 50.0), cudahm.EINVAL),
    (lambda c: [setattr(c, "model", cudahm.NN3), setattr(c, "d", 3)] and None, cudahm.EINVAL),  # C_pop = 0
    (lambda c: [setattr(c, "model", cudahm.NN3), setattr(c, "d", 3),
                [c.model_consts.__setitem__(q, v) for q, v in enumerate((1.0, 2.0, 1.0, 0.0, 0.0, 1.0))]] and None,
     cudahm.EINVAL),  # C_pop not positive definite
    (lambda c: setattr(c, "marginal", 2), cudahm.EINVAL),
    (lambda c: [setattr(c, "marginal", 1), setattr(c, "model", cudahm.NN3), setattr(c, "d", 3),
                [c.model_consts.__setitem__(q, v) for q, v in enumerate((1.0, 0.0, 1.0, 0.0, 0.0, 1.0))]] and None,
     cudahm.EUNSUPPORTED),  # the marginal form integrates 1-D latents only
    (lambda c: setattr(c, "keep_chi_moments", 3), cudahm.EINVAL),
    (lambda c: [setattr(c, "keep_chi_moments", 1), setattr(c, "marginal", 1)] and None,
     cudahm.EINVAL),  # the marginal form has no latents
])
def test_invalid_configs_rejected(lib, mutate, code):
    cfg = cudahm.cudahm_config_init(cudahm.NN1, 100)
    mutate(cfg)
    with pytest.raises(cudahm.CudahmError) as ei:
        cudahm.cudahm_create(cfg)
    assert ei.value.code == code
    assert len(str(ei.value)) > 10


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(cudahm, "_lib", None)
    monkeypatch.setattr(cudahm, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        cudahm.lib()
