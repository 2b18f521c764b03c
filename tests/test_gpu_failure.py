"""Failure detection without a GPU fault: a bounded wait on a flag nothing
sets reports TIMEOUT through the device status word, and an allocation
failure injected on the host comes back as GMGM_E_NOMEM; in both cases the
handle stays usable."""

import numpy as np
import pytest
import torch

from oracle import gram as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g(cuda_dev):
    import paper_2407_19892_gb300 as pkg
    from paper_2407_19892_gb300 import build
    build.build()
    return pkg


def test_bounded_wait_gives_up_with_timeout_status(g, cuda_dev):
    h = g.Handle(cuda_dev)
    assert h.device_status() == 0
    h.probe_wait(1000)
    assert h.device_status() & 0x10  # GMGM_DEV_TIMEOUT
    assert h.device_status() == 0    # read and cleared
    # the context and the handle keep working
    x = np.random.default_rng(1).standard_normal((300, 40)).astype(np.float32)
    S = g.gram(torch.from_numpy(x).to(cuda_dev), g.SIDE_COLS, g.FP32, h=h).cpu().numpy()
    ref = og.gram(x.astype(np.float64), 1)
    assert np.max(np.abs(S - ref)) <= 2e-6 * np.abs(ref).max()
    assert h.device_status() == 0
    with pytest.raises(g.GmgmError):
        h.probe_wait(0)


def test_injected_allocation_failure(g, cuda_dev, monkeypatch):
    S = torch.diag(torch.arange(1, 51, dtype=torch.float64)).to(cuda_dev)
    monkeypatch.setenv("GMGM_FAULT", "alloc")
    h = g.Handle(cuda_dev)  # fresh handle: its scratch has to grow
    with pytest.raises(g.GmgmError) as ei:
        g.spectra(S, 50, h=h)
    assert ei.value.code == -3  # GMGM_E_NOMEM
    monkeypatch.delenv("GMGM_FAULT")
    ev, _ = g.spectra(S, 50, h=h)
    np.testing.assert_allclose(ev.cpu().numpy(), np.arange(50, 0, -1, dtype=np.float64), rtol=0, atol=1e-11 * 50)
