"""GPU parity of the exact-ray horizontal constants (FLIC_FLAG_EXACT_RAY): tables, edge
bits and labels against the oracle's exact-ray tables, element by element."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2003_00575_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


def _run(flic, rng, elev, az, delta, skip, wrap, tuning=None):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap, exact_ray=True)
    try:
        if tuning:
            flic.flic_set_tuning(h, *tuning)
        kv, kh = flic.flic_get_tables(h)
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        lab = torch.full((R * C,), 12345, dtype=torch.int32, device=DEV)
        m = torch.zeros(R * C, dtype=torch.int16, device=DEV)
        flic.flic_label(h, r, lab)
        flic.flic_edges(h, r, m)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        return kv, kh, lab.cpu().numpy().reshape(R, C), m.cpu().numpy().view(np.uint16).reshape(R, C)
    finally:
        h.close()


def _check(flic, rng, elev, az, delta, skip, wrap=True, tuning=None):
    kv, kh, lab, m = _run(flic, rng, elev, az, delta, skip, wrap, tuning)
    okv, okh = oracle.tables(elev, az, skip, exact_ray=True)
    np.testing.assert_array_equal(kv, okv)
    np.testing.assert_array_equal(kh, okh)
    np.testing.assert_array_equal(m, oracle.edges(rng, elev, az, delta, skip, wrap, exact_ray=True))
    np.testing.assert_array_equal(lab, oracle.label(rng, elev, az, delta, skip, wrap,
                                                    exact_ray=True))


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_configs(flic, name):
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[name]()
    _check(flic, f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)


@pytest.mark.parametrize("seed", range(12))
def test_random(flic, seed):
    g = np.random.default_rng(500 + seed)
    R, C, S = int(g.integers(2, 60)), int(g.integers(8, 600)), int(g.integers(1, 9))
    elev = np.radians(np.sort(g.uniform(-45, 45, R))[::-1])
    rng = (8 + g.normal(0, 0.05, (R, C))).astype(np.float32)
    rng[g.random((R, C)) < 0.2] = 0
    tuning = [(0, 0, 0), (64, 128, 64), (512, 256, 8)][seed % 3]
    _check(flic, rng, elev, 2 * math.pi / C, float(g.uniform(0.05, 0.5)), S,
           bool(seed % 2), tuning)
