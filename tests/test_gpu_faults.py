"""Failure paths on the GPU, injected from the host (no trap, no hang).

SBR_FAULT=alloc: every library allocation reports failure; the call returns
SBR_ERR_ALLOC and the process keeps working once the variable is cleared.
SBR_FAULT=timeout: the tensor-core synthesis waits on an mbarrier that nothing
arrives at; the bounded wait gives up, the kernel records SBR_ERR_TIMEOUT,
frees its tensor memory and returns; sbr_path_query reports it, and the
context stays usable.
"""
import os

import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_10006_gb300 import build as b
    b.build()
    import paper_2208_10006_gb300 as m
    return m


@pytest.fixture
def fault():
    def set_(mode):
        os.environ["SBR_FAULT"] = mode
    yield set_
    os.environ.pop("SBR_FAULT", None)


def test_injected_allocation_failure(sbr, fault):
    d = sbr.scene_to_device(scenes.config1(N=20, K=2))
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    fault("alloc")
    with pytest.raises(sbr.SbrError) as e:
        sbr.trace(bvh, d["tx"], d["rx"], 20, 2)
    assert e.value.status == 8
    os.environ.pop("SBR_FAULT")
    tr = sbr.trace(bvh, d["tx"], d["rx"], 20, 2)
    assert sbr.paths(tr, bvh).n >= 1


def test_injected_barrier_timeout_is_reported_and_recoverable(sbr, fault):
    sc = scenes.config3(N=30, K=2, F=4, ny_tx=4, nz_tx=4, n_rx=8)
    r = sbr.run_scene(sc)
    d = r["dev"]
    fault("timeout")
    sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, sbr.SYNTH_BF16X3)
    with pytest.raises(sbr.SbrError) as e:
        r["paths"].info()
    assert e.value.status == 5
    os.environ.pop("SBR_FAULT")
    # the context is intact: a fresh path list synthesises normally
    r2 = sbr.run_scene(sc)
    H64 = sbr.synthesize_H(r2["paths"], r2["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, 0)
    Htc = sbr.synthesize_H(r2["paths"], r2["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, 2)
    assert r2["paths"].info()["status"] == 0
    H64, Htc = H64.cpu().numpy(), Htc.cpu().numpy()
    assert np.abs(Htc - H64).max() < 5e-5 * np.abs(H64).max()
