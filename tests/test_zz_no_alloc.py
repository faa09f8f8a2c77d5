"""The allocation-free smoother entry point agrees with the regular one.

dpgmg_smooth_noalloc serves callers that cannot let the library allocate
device memory (their memory is pre-reserved by their own arena, or their
loop cannot take the synchronisation of cudaMalloc/cudaFree): its scratch is
a fixed array compiled into the library.  Here it is called through the C ABI
on device buffers, twice in a row on different inputs per level (the second
call reuses the array the first one left behind), and compared with
dpgmg_apply(DPGMG_OP_SMOOTH) at the tolerances of the other parity tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-6)])
def test_noalloc_smoother_matches_regular_entry_point(precision, tol):
    torch = pytest.importorskip("torch")
    from paper_2304_01728_gb300 import dpgmg as D

    # 4^3 p2 -> 4^3 p1 -> 2^3 p1: one p-level and one h-level smoother
    pk = dict(n=(4, 4, 4), p=2, omega=5.0, src_center=(0.4, 0.5, 0.6), src_width=0.15)
    with D.Solver(pk, n_levels=3, p_min=1, precision=precision) as s:
        for level in (1, 2):
            n = s.level(level).n_dof
            for call in range(2):
                x = _rand(n, 100 * level + call)
                ref = D.dpgmg_apply(s.h, s.s, D.OP_SMOOTH, level, x, n)
                xd = torch.from_numpy(x.view(np.float64).copy()).to("cuda")
                yd = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                D.dpgmg_smooth_noalloc(s.h, s.s, level, xd.data_ptr(), yd.data_ptr())
                y = yd.cpu().numpy().view(np.complex128)
                assert np.all(np.isfinite(y))
                assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol, (level, call)
        # a level without a smoother is rejected
        xd = torch.zeros(2 * s.level(0).n_dof, dtype=torch.float64, device="cuda")
        with pytest.raises(D.DpgmgError) as e:
            D.dpgmg_smooth_noalloc(s.h, s.s, 0, xd.data_ptr(), xd.data_ptr())
        assert e.value.code == D.DPGMG_ERR_ARG
