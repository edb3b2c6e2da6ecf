"""The large workload: a procedural city of 2,015,232 triangles (64 x 64 buildings
and a ground grid), 256 sources, 8 bands, 200 reflections, IR 3 s at 1 kHz, SH
order 3, through the launch configuration bench.py --workload large times (device
positions).  Element-by-element parity against the oracle on 50,000 primaries of
the full scene; at the full million primaries, the outputs the oracle computes one
by one (direct sound of all 256 sources) and the properties that hold at any size."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1803_00430_gb300 import rpr, scenes  # noqa: E402

import oracle  # noqa: E402
import parity_util as pu  # noqa: E402

LARGE = dict(max_order=200, sh_order=3, num_bins=3000, min_order=1, ir_rate_hz=1000.0,
             seed=scenes.PHILOX_KEY_BASE + 4)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = rpr.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def city():
    return scenes.city()


@pytest.fixture(scope="module")
def city_scene(ctx, city):
    return rpr.Scene.from_scene(ctx, city)


def _gpu(ctx, sc, scene, p, want_hash):
    import ctypes
    q = rpr.TraceParams(**{**p.__dict__})
    q.flags |= rpr.RP_FLAG_DEVICE_POSITIONS | (rpr.RP_FLAG_RAY_HASH if want_hash else 0)
    out = rpr.DeviceTrace(sc.num_sources, sc.num_bands, q.K, q.num_bins, want_hash=q.num_rays if want_hash else 0)
    lis = torch.tensor(sc.listener, device="cuda")
    src = torch.tensor(sc.sources, device="cuda")
    rpr.check(ctx.lib.rp_trace(scene.h, ctypes.byref(q.c()), rpr._ptr(lis), rpr._ptr(src), sc.num_sources,
                               rpr._ptr(out.H), rpr._ptr(out.direct), rpr._ptr(out.stats),
                               rpr._ptr(out.ray_hash) if want_hash else None), "rp_trace")
    rpr.check(ctx.sync_status(), "rp_trace")
    prm = rpr.estimate(ctx, out.H, out.direct, q.ir_rate_hz)
    return {"H": out.H.double().cpu().numpy(), "stats": out.stats_dict(), "direct": out.direct_dict(),
            "hash": out.hashes()[: q.num_rays] if want_hash else None,
            "params": rpr.params_to_dict(prm.cpu().numpy().tobytes(), sc.num_sources, sc.num_bands, q.K)}


def test_city_parity_50k_primaries(ctx, city, city_scene):
    p = rpr.TraceParams(num_rays=50_000, **LARGE)
    g = _gpu(ctx, city, city_scene, p, want_hash=True)
    o = pu.run_oracle(city, p, threads=os.cpu_count())
    assert g["stats"]["error"] == 0
    assert g["stats"]["segments"] == o["stats"]["segments"]
    assert np.abs(o["H"]).sum() > 0
    rep = pu.assert_parity(g, o, p.num_rays, check_params=False)
    # At 50k primaries many of the 2048 (source, band) IRs of a city are sparse; where
    # the fit window or a near-flat fit turns on rounding-level differences of H the
    # parameters are ill-posed (the estimator itself is pinned on identical H).  The
    # 0.5 % bar holds on the well-posed fits: the same window on both sides, at least
    # 20 bins, R^2 >= 0.9.
    rep.update(pu.assert_well_posed_params(g, o, min_well=50, min_kinds_equal=0.95))
    print("city, 50k primaries:", rep, "segments", g["stats"]["segments"], "shadow rays", g["stats"]["shadow_rays"])


def test_city_full_size_direct_and_invariants(ctx, city, city_scene):
    p = rpr.TraceParams(num_rays=1_000_000, **LARGE)
    g = _gpu(ctx, city, city_scene, p, want_hash=False)
    st = g["stats"]
    assert st["error"] == 0 and st["primaries"] == p.num_rays
    assert 0 < st["segments"] <= p.num_rays * p.max_order
    H = g["H"]
    assert np.isfinite(H).all() and (H[:, :, 0] >= 0).all()
    # per ray and band, every unit of weight ends escaped, absorbed or remaining; the
    # per-band reweighting of the continuation keeps this only in expectation
    total = np.array(st["escaped"]) + np.array(st["absorbed"]) + np.array(st["remaining"])
    np.testing.assert_allclose(total[:city.num_bands] / p.num_rays, 1.0, rtol=0.02)
    # direct sound of all 256 sources, which the oracle computes one by one
    osc = oracle.OracleScene.from_scene(city)
    od = oracle.direct(osc, pu.oracle_params(p), city.listener, city.sources)
    np.testing.assert_array_equal(g["direct"]["visible"], od["visible"])
    np.testing.assert_array_equal(g["direct"]["bin"], od["bin"])
    np.testing.assert_allclose(g["direct"]["energy"], od["energy"], rtol=1e-6)
    print("city, 1M primaries: segments", st["segments"], "shadow rays", st["shadow_rays"],
          "visible sources", int(np.sum(od["visible"])))
