"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/hbugks.h declares, and
its host-side validation rejects invalid cases (no GPU compute is called)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_03479_gb300 import build, hbugks, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return hbugks.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hbugks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hbugks_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(hbugks.EXPORTED)


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)


def test_status_strings(L):
    assert hbugks.status_string(0) == "ok"
    assert hbugks.status_string(-4) == "diverged"
    assert hbugks.status_string(123) == "unknown status"


def test_workspace_size_and_validation(L):
    c = I.config1()
    n = hbugks.workspace_bytes([c])
    # state: 2 buffers x (h, b) x nt * nc * nvel doubles, plus W and tables
    assert n > 4 * c.nt * c.nc * c.nvel * 8
    c32 = I.config1()
    c32.precision = 1
    assert hbugks.workspace_bytes([c32]) < n
    bad = I.config1()
    bad.xnodes = bad.xnodes[::-1].copy()              # decreasing nodes
    assert hbugks.workspace_bytes([bad]) == 0
    bad = I.config1()
    bad.n_harmonics = 8                                # N_T = 17 > 15
    assert hbugks.workspace_bytes([bad]) == 0
    bad = I.config1()
    bad.walls[2][2] = -1.0                             # negative wall temperature
    assert hbugks.workspace_bytes([bad]) == 0
    mixed = [I.config1(), c32]                         # one handle, one precision
    assert hbugks.workspace_bytes(mixed) == 0
    assert hbugks.workspace_bytes(I.config4_cases()) > 0


def test_time_domain_mode_needs_one_level_and_a_frequency():
    from paper_2605_03479_gb300 import hbugks as hb
    from paper_2605_03479_gb300 import inputs as I
    c = I.make_case("td", 5, 8, kn=0.1, st=1.0, nh=0, drive="shear")
    c.td_steps = 40
    assert hb.workspace_bytes([c]) > 0
    c.n_harmonics = 1
    assert hb.workspace_bytes([c]) == 0
    c.n_harmonics, c.st = 0, 0.0
    assert hb.workspace_bytes([c]) == 0
    c.st, c.td_steps = 1.0, -1
    assert hb.workspace_bytes([c]) == 0


@pytest.mark.parametrize("spoil", [
    lambda c: c.u.__setitem__(3, np.nan),                  # a velocity node
    lambda c: c.wv.__setitem__(0, np.inf),                 # a weight
    lambda c: c.xnodes.__setitem__(-1, np.inf),            # the last mesh node
    lambda c: setattr(c, "kn", np.inf),
    lambda c: setattr(c, "st", np.nan),
    lambda c: setattr(c, "cfl", np.inf),
    lambda c: setattr(c, "pr", 0.0),
    lambda c: setattr(c, "umax", 0.0),
    lambda c: c.walls[2].__setitem__(3, np.nan),           # the lid amplitude
], ids=["nan_node", "inf_weight", "inf_mesh_node", "inf_kn", "nan_st", "inf_cfl", "zero_pr", "zero_umax",
        "nan_wall"])
def test_non_finite_inputs_are_rejected(L, spoil):
    c = I.config1()
    assert hbugks.workspace_bytes([c]) > 0
    spoil(c)
    assert hbugks.workspace_bytes([c]) == 0


def test_cases_beyond_32_bit_table_offsets_are_rejected(L):
    # 3000 x 3000 cells, 16 x 16 velocities, N_T = 15: the per-cell expm1 table [nc][nt][2][nu + nv] would hold
    # 8.6e9 elements (its state, 552 GB, would not fit in HBM either); 1000 x 1000 cells keep it at 9.6e8
    big = I.make_case("big", 3000, 16, kn=0.1, st=1.0, nh=7, drive="shear")
    assert hbugks.workspace_bytes([big]) == 0
    ok = I.make_case("ok", 1000, 16, kn=0.1, st=1.0, nh=7, drive="shear")
    assert hbugks.workspace_bytes([ok]) > 0
