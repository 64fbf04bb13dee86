"""The autotuner cache on the GPU: the first autotune of a problem times the
candidates and records the winner, a second handle with the same key applies
the recorded shape without timing (a hit), and the recorded run steps to the
same bits as a run with that shape set by hand."""
import numpy as np
import pytest

from paper_2005_08674_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm as m
    return m


def test_single_domain_choice_is_recorded_and_reused(lbm, tmp_path):
    path = tmp_path / "tune.json"
    lbm.lbm_set_tune_cache(str(path))
    try:
        w = inputs.pulse_200()
        h0, m0 = lbm.lbm_tune_cache_stats()
        with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as a:
            a.init(*w.fields())
            first = a.autotune()
            shape_a = (a.staged, a.fused)
            a.step(40)
            ref = a.populations()
        assert lbm.lbm_tune_cache_stats() == (h0, m0 + 1)
        assert path.exists() and "domain" in path.read_text()
        with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as b:
            b.init(*w.fields())
            second = b.autotune()
            assert (b.staged, b.fused) == shape_a
            b.step(40)
            got = b.populations()
        assert lbm.lbm_tune_cache_stats() == (h0 + 1, m0 + 1)
        assert second[:3] == first[:3] and second[3] == pytest.approx(first[3])
        assert np.array_equal(got, ref)
        # another storage is another key
        with lbm.Simulation(w.nx, w.ny, w.tau, storage="f16") as c:
            c.init(*w.fields())
            c.autotune()
        assert lbm.lbm_tune_cache_stats() == (h0 + 1, m0 + 2)
    finally:
        lbm.lbm_set_tune_cache(None)


def test_batch_choice_is_recorded_and_reused(lbm, tmp_path):
    path = tmp_path / "tune.json"
    lbm.lbm_set_tune_cache(str(path))
    try:
        ws = inputs.batch_instances(count=6, lo=16, hi=120)
        h0, m0 = lbm.lbm_tune_cache_stats()
        with lbm.Batch(ws, storage="f32") as a:
            for k, w in enumerate(ws):
                a.init(k, *w.fields())
            first = a.autotune()
        with lbm.Batch(ws, storage="f32") as b:
            for k, w in enumerate(ws):
                b.init(k, *w.fields())
            second = b.autotune()
        assert lbm.lbm_tune_cache_stats() == (h0 + 1, m0 + 1)
        assert second[:6] == first[:6]
    finally:
        lbm.lbm_set_tune_cache(None)


def test_malformed_cache_falls_back_to_timing(lbm, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{ this is not the cache format")
    lbm.lbm_set_tune_cache(str(path))
    try:
        w = inputs.pulse_200()
        h0, m0 = lbm.lbm_tune_cache_stats()
        with lbm.Simulation(w.nx, w.ny, w.tau, storage="f32") as a:
            a.init(*w.fields())
            a.autotune()
        assert lbm.lbm_tune_cache_stats() == (h0, m0 + 1)
        assert path.read_text().startswith('{"lbm_tune_cache": 1')
    finally:
        lbm.lbm_set_tune_cache(None)
