"""C-ABI library: builds for sm_103a, loads, exports every declared symbol,
and its host-only entry points agree with the paper's formulas (no GPU)."""
import ctypes as C
import math
import os
import re

import pytest

import oracle
from paper_2105_10576_gb300 import build as gbuild
from paper_2105_10576_gb300 import inputs, oscar

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return oscar.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "oscar.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(oscar_\w+)\s*\(", txt, re.M)))


def test_header_declares_binding_exports():
    assert declared_symbols() == sorted(oscar.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_targets_sm103a(lib):
    # the cubin is built for sm_103a only (checked through the build flags)
    assert "arch=compute_103a,code=sm_103a" in " ".join(gbuild.ARCH)


def test_strerror(lib):
    assert lib.oscar_strerror(0) == b"ok"
    assert lib.oscar_strerror(-1) == b"invalid argument"


@pytest.mark.parametrize("case", ["bubble", "constriction", "micromodel"])
def test_timesteps_match_oracle(lib, case):
    c = {"bubble": lambda: inputs.channel_bubble_2d(),
         "constriction": lambda: inputs.constricted_channel_3d(nx=16, ny=8, nz=8),
         "micromodel": lambda: inputs.micromodel_2d(nx=64, ny=32)}[case]()
    cc = c.meta["c_cfl"]
    for solid in (None, c.solid):
        a = oscar.oscar_timesteps(c.params, cc, solid)
        b = oracle.timesteps(c.params, cc, solid)
        for x, y in zip(a[:3], b[:3]):
            assert x == pytest.approx(y, rel=1e-15)
        assert a[3] == b[3]


def test_timesteps_reject_a_blocked_channel(lib):
    """A column with no fluid while the inlet has some: no path to the outlet."""
    c = inputs.channel_bubble_2d(nx=16, ny=4)
    s = c.solid.copy()
    s[:, 7] = 1
    with pytest.raises(oscar.OscarError):
        oscar.oscar_timesteps(c.params, 0.1, s)
    with pytest.raises(ValueError):
        oracle.timesteps(c.params, 0.1, s)


def test_create_rejects_bad_arguments(lib):
    p = inputs.default_params(dim=4)
    P = oscar.make_params(p)
    h = C.c_void_p()
    rc = lib.oscar_create(C.byref(P), None, None, None, C.byref(h))
    assert rc == -1 and not h.value
    assert lib.oscar_drag_step(None, 1.0) == -1
    assert lib.oscar_relax(None, 1.0, 3, None, None) == -1


def test_footprint_is_host_only_and_scales(lib):
    """oscar_footprint computes the arena size without a GPU: it grows with the
    grid, and the FP64 path needs more than the mixed path."""
    c = inputs.constricted_channel_3d(nx=64, ny=16, nz=16)
    mixed = oscar.oscar_footprint(dict(c.params, precision=inputs.PREC_MIXED))
    fp64 = oscar.oscar_footprint(dict(c.params, precision=inputs.PREC_FP64))
    big = oscar.oscar_footprint(dict(inputs.constricted_channel_3d(nx=128, ny=32, nz=32).params,
                                     precision=inputs.PREC_MIXED))
    n = 64 * 16 * 16
    assert 50 * n < mixed < fp64 < 2000 * n
    assert 7 * mixed < big < 9 * mixed
    with pytest.raises(oscar.OscarError):
        oscar.oscar_footprint(dict(c.params, nx=0))
