"""Sampling-rate tuning by the autocorrelation time of the mean psi_6 (the
criterion of Sec. 3.3), in a liquid where that time is short."""
import pytest

from paper_1211_1646_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1211_1646_gb300 import build
    build.build()


def test_tune_sampling_ranks_candidates_by_tau_per_second():
    from paper_1211_1646_gb300 import hdmc
    from paper_1211_1646_gb300.analysis import tune_sampling
    nx, ny = W.hex_counts(4096)
    Lx, Ly = W.hex_box(nx, ny, 0.50)

    def make(d, nm):
        return hdmc.System(nx * ny, Lx, Ly, 1.0, d, nm, 17, "fp32")

    res = tune_sampling(make, [(0.05, 4), (0.25, 4)], sweeps=40000, every=10, equilibrate=2000)
    by_d = {r["d"]: r for r in res}
    print(res)
    assert [r["tau_seconds"] for r in res] == sorted(r["tau_seconds"] for r in res)
    # small moves decorrelate psi_6 more slowly per sweep
    assert by_d[0.05]["tau_sweeps"] > 2 * by_d[0.25]["tau_sweeps"]
    assert all(r["seconds_per_sweep"] > 0 for r in res)
