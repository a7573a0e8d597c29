"""The no-allocation harmonic entry point (hbugks_harmonic_noalloc) against the handle-based one.

Some callers cannot allocate device memory (they run under an allocator they do not control, or the
device memory is already fully handed out), so they cannot give a handle its workspace.  The entry point
takes a state that already lives in device memory and keeps its intermediates in a fixed array inside the
library.  This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2605_03479_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_harmonic_matches_handle_on_two_calls():
    import torch
    from paper_2605_03479_gb300 import build, hbugks as hb
    build.build()
    case = I.make_case("na", 7, 10, kn=0.2, st=1.0, nh=2, pr=2 / 3, drive="thermal", amp=0.3, ncell_y=6)
    s = hb.Solver(case)
    s.set_state(0, *I.initial_state(case, seed=9))
    s.iterate(4)
    W, h, b = s.get_state(0)
    expected = [s.harmonic(0, k) for k in range(case.n_harmonics + 1)]
    s.destroy()
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    du, dwu, dv, dwv, dh, db = t(case.u), t(case.wu), t(case.v), t(case.wv), t(h), t(b)
    for call in range(2):                       # the fixed array keeps the previous call's contents
        for k in range(case.n_harmonics + 1):
            re = torch.full((8, case.nc), np.nan, dtype=torch.float64, device=dev)
            im = torch.full((8, case.nc), np.nan, dtype=torch.float64, device=dev)
            rc = hb.harmonic_noalloc(case.nx, case.ny, case.nu, case.nv, du, dwu, dv, dwv, case.nt, dh, db, k, re, im)
            assert rc == hb.OK
            torch.cuda.synchronize()
            got = re.cpu().numpy() + 1j * im.cpu().numpy()
            np.testing.assert_allclose(got, expected[k], rtol=1e-9, atol=1e-12)


def test_noalloc_harmonic_rejects_sizes_beyond_its_array():
    import torch
    from paper_2605_03479_gb300 import build, hbugks as hb
    build.build()
    dev = torch.device("cuda:0")
    one = torch.zeros(4, dtype=torch.float64, device=dev)
    nx = ny = 128                                # 8 * 5 levels * 128 * 128 > 2^19 doubles
    rc = hb.harmonic_noalloc(nx, ny, 2, 2, one, one, one, one, 5, one, one, 0, one, one)
    assert rc == hb.EINVAL
    rc = hb.harmonic_noalloc(4, 4, 2, 2, one, one, one, one, 5, one, one, 3, one, one)   # k > N_H
    assert rc == hb.EINVAL
