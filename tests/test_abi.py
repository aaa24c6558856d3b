"""The C-ABI library without a GPU: it loads, exports every function that
include/gce.h declares, and its host-side argument checks accept and reject
what the header says.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2006_06866_gb300 as g
from paper_2006_06866_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gce.h")


@pytest.fixture(scope="module")
def L():
    from paper_2006_06866_gb300 import build
    build.build()
    return g.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gce_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_bound_symbols():
    decl = declared_functions()
    assert decl == sorted(binding.SIGNATURES), (decl, sorted(binding.SIGNATURES))


def test_header_constants_match_the_binding():
    """Every #define GCE_* and enum value of the header has the binding's value."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"#define\s+(GCE_[A-Z_0-9]+)\s+(\d+)u?\b", text)}
    consts.update({k: int(v) for k, v in re.findall(r"\b(GCE_[A-Z_0-9]+)\s*=\s*(\d+)", text)})
    assert len(consts) >= 14, consts
    for name, value in consts.items():
        assert getattr(binding, name) == value, name
        assert getattr(g, name) == value, name


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_status_strings(L):
    for s in range(5):
        assert L.gce_status_string(s)
    assert L.gce_status_string(99) == b"unknown status"


def _ok(offsets, n_p=10, n_q=1, k=0, **cfg):
    c = g.Config(**cfg)
    return g.gce_check_job(np.asarray(offsets, dtype=np.int64), n_p, n_q, c, k)


def test_check_job_accepts_valid_jobs(L):
    assert _ok([0, 5, 9]) == g.GCE_OK
    assert _ok([0, 65535]) == g.GCE_OK
    assert _ok([0, 1], n_p=3, n_q=2, k=6) == g.GCE_OK
    assert _ok([0], n_p=1) == g.GCE_OK  # empty batch
    for mode in ("fp64", "split32", "fixed32"):
        assert _ok([0, 3], phase_mode=mode, n_phase_bins=256, n_mag_bins=255) == g.GCE_OK


@pytest.mark.parametrize("case", [
    dict(offsets=[1, 5]),                    # does not start at 0
    dict(offsets=[0, 5, 4]),                 # decreasing
    dict(offsets=[0, 5, 5]),                 # empty curve
    dict(offsets=[0, 65536]),                # longer than the maximum
    dict(offsets=[0, 5], n_p=0),
    dict(offsets=[0, 5], n_q=0),
    dict(offsets=[0, 5], n_p=70000, n_q=70000),  # >= 2^32 trials
    dict(offsets=[0, 5], k=-1),
    dict(offsets=[0, 5], k=65),
    dict(offsets=[0, 5], n_p=3, k=4),        # more than the grid holds
    dict(offsets=[0, 5], n_phase_bins=0),
    dict(offsets=[0, 5], n_phase_bins=257),
    dict(offsets=[0, 5], n_mag_bins=0),
    dict(offsets=[0, 5], n_mag_bins=256),
    dict(offsets=[0, 5], phase_mode=7),
    dict(offsets=[0, 5], t0=float("nan")),
])
def test_check_job_rejects(L, case):
    assert _ok(**case) == g.GCE_ERR_INVALID


def test_loading_fails_loudly_without_the_library(monkeypatch):
    monkeypatch.setattr(binding, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        binding.lib()


def test_binding_rejects_arrays_on_different_devices():
    """The binding's device check (no GPU needed: stand-ins carry only a device):
    every array of a call must share one CUDA device, and that device must be the
    handle's when a handle is given."""
    from types import SimpleNamespace as NS

    import torch

    from paper_2006_06866_gb300.binding import one_device

    def on(i):
        return NS(device=torch.device("cuda", i))

    assert one_device([("times", on(1)), ("mags", on(1)), ("out", None)]) == 1
    assert one_device([("times", on(0)), ("mags", on(0))], device=0) == 0
    with pytest.raises(ValueError, match="mags is on cuda:1"):
        one_device([("times", on(0)), ("mags", on(1))])
    with pytest.raises(ValueError, match="handle on cuda:0"):
        one_device([("times", on(1)), ("mags", on(1))], device=0)
