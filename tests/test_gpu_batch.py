"""Many uneven systems in one persistent launch, against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-4  # FP32 arithmetic: n eps32 kappa for n <= 1024, kappa ~ 1.5


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=dtype).T)).cuda().t()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _systems(count, nmax, kmax, seed, dtype=np.float64, n0s=(32, 64)):
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.rint(np.exp(rng.uniform(np.log(1), np.log(nmax)))))
        k = int(np.rint(np.exp(rng.uniform(np.log(1), np.log(kmax)))))
        L, B = inputs.well_conditioned(n, k, seed=seed * 1000 + i)
        out.append({"Lh": L, "Bh": B, "L": _dev(L, dtype), "B": _dev(B, dtype),
                    "X": torch.full((k, n), float("nan"), dtype=torch.float64 if dtype == np.float64
                                    else torch.float32, device="cuda").t(),
                    "n0": n0s[i % len(n0s)]})
    return out


def test_batch_fp64_uneven(cuda_lib):
    import paper_1612_01855_gb300 as g
    systems = _systems(60, 300, 70, seed=1)
    batch = g.Batch(systems)
    batch.run()
    rc, item, row = batch.status()
    assert rc == 0
    for sy in systems:
        want = oracle.forward_subst(sy["Lh"], sy["Bh"])
        assert _rel(sy["X"].cpu().numpy(), want) < TOL64


def test_batch_fp32_uneven(cuda_lib):
    import paper_1612_01855_gb300 as g
    systems = _systems(40, 400, 50, seed=2, dtype=np.float32)
    batch = g.Batch(systems, dtype="f32")
    batch.run()
    assert batch.status()[0] == 0
    for sy in systems:
        want = oracle.forward_subst(sy["Lh"].astype(np.float32).astype(np.float64),
                                    sy["Bh"].astype(np.float32).astype(np.float64))
        assert _rel(sy["X"].cpu().numpy().astype(np.float64), want) < TOL32


def test_batch_fp32_large_and_wide(cuda_lib):
    """FP32 systems up to n = 1024 and k = 256 (many column chunks per
    system), with n not a multiple of n0 and k not a multiple of the chunk."""
    import paper_1612_01855_gb300 as g
    systems = _systems(10, 1024, 256, seed=12, dtype=np.float32)
    systems[0] = _systems(1, 2, 2, seed=13, dtype=np.float32)[0]  # n, k tiny
    for sy in systems[1:4]:
        sy["n0"] = 64
    batch = g.Batch(systems, dtype="f32")
    batch.run()
    assert batch.status()[0] == 0
    for sy in systems:
        want = oracle.forward_subst(sy["Lh"].astype(np.float32).astype(np.float64),
                                    sy["Bh"].astype(np.float32).astype(np.float64))
        assert _rel(sy["X"].cpu().numpy().astype(np.float64), want) < TOL32


def test_batch_fp32_tiles_mix_and_graph_are_bitwise_stable(cuda_lib):
    """Every FP32 output is summed in one fixed order: 8-, 16- and 32-wide
    column chunks give the same bits, a system alone equals the system in the
    mix, and a captured graph replays the same bits."""
    import torch
    import paper_1612_01855_gb300 as g
    systems = _systems(20, 600, 70, seed=9, dtype=np.float32)
    ref = None
    for tile in (0, 8, 16, 32):
        for sy in systems:
            sy["tile_cols"] = tile
            sy["X"].fill_(float("nan"))
        b = g.Batch(systems, dtype="f32")
        b.run()
        assert b.status()[0] == 0
        got = [sy["X"].clone() for sy in systems]
        if ref is None:
            ref = got
        else:
            assert all(torch.equal(a, c) for a, c in zip(ref, got)), tile
    for i in (2, 11):
        alone = dict(systems[i])
        alone["X"] = torch.empty_like(systems[i]["X"].t()).t()
        b = g.Batch([alone], dtype="f32")
        b.run()
        assert b.status()[0] == 0
        assert torch.equal(alone["X"], ref[i])
    b = g.Batch(systems, dtype="f32")
    b.capture()
    for sy in systems:
        sy["X"].fill_(float("nan"))
    b.launch_graph()
    b.launch_graph()
    assert b.status()[0] == 0
    assert all(torch.equal(sy["X"], x0) for sy, x0 in zip(systems, ref))


@pytest.mark.parametrize("n0", [None, 32, 64])
def test_batch_fp32_reports_singular_item(cuda_lib, n0):
    """A zero pivot is reported by the first failing item and its row; a
    later failing item does not hide it.  n0 = 32: the warp-per-block
    inversions; 64: the CTA-per-block RecTriInv; None: both in one batch."""
    import paper_1612_01855_gb300 as g
    systems = _systems(8, 200, 40, seed=5, dtype=np.float32, n0s=(32, 64) if n0 is None else (n0,))
    bad = next(i for i in range(2, 7) if systems[i]["Lh"].shape[0] >= 4)
    r = systems[bad]["Lh"].shape[0] // 2
    systems[bad]["L"][r, r] = 0.0
    systems[7]["L"][0, 0] = 0.0
    b = g.Batch(systems, dtype="f32")
    b.run()
    rc, item, row = b.status()
    assert rc == -2 and item == bad and row == r


def test_batch_fp32_n0_32_two_block_steps(cuda_lib):
    """n0 = 32: the units walk 64-row steps of two blocks (the second
    block's update by the first in between); sizes that end a step after
    one block, in the middle of the second, or on a step boundary, and
    narrow and wide column chunks, against the oracle and against n0 = 64."""
    import torch
    import paper_1612_01855_gb300 as g
    shapes = [(32, 5), (33, 40), (64, 17), (95, 64), (96, 33), (128, 8), (129, 100), (500, 256), (1000, 31)]
    got = {}
    for n0 in (32, 64):
        systems = []
        for i, (n, k) in enumerate(shapes):
            L, B = inputs.well_conditioned(n, k, seed=4200 + i)
            systems.append({"Lh": L, "Bh": B, "L": _dev(L, np.float32), "B": _dev(B, np.float32),
                            "X": torch.full((k, n), float("nan"), dtype=torch.float32, device="cuda").t(),
                            "n0": n0})
        b = g.Batch(systems, dtype="f32")
        b.run()
        assert b.status()[0] == 0
        got[n0] = [sy["X"].cpu().numpy().astype(np.float64) for sy in systems]
        for sy, x in zip(systems, got[n0]):
            want = oracle.forward_subst(sy["Lh"].astype(np.float32).astype(np.float64),
                                        sy["Bh"].astype(np.float32).astype(np.float64))
            assert _rel(x, want) < TOL32, (n0, sy["Lh"].shape[0])
    for a, c in zip(got[32], got[64]):
        assert _rel(a, c) < 2 * TOL32


def test_batch_with_resident_plans_and_graph(cuda_lib):
    """Items with resident plans (any n0) next to plan-less items; a captured
    CUDA graph replays the same results."""
    import torch
    import paper_1612_01855_gb300 as g
    systems = _systems(12, 700, 90, seed=3)
    plans = []
    for i, sy in enumerate(systems):
        if i % 2 == 0:
            p = g.trsm_plan(sy["L"], [32, 100, 256][i % 3])
            plans.append(p)
            sy["plan"] = p
    batch = g.Batch(systems)
    batch.run()
    assert batch.status()[0] == 0
    first = [sy["X"].clone() for sy in systems]
    for sy in systems:
        want = oracle.forward_subst(sy["Lh"], sy["Bh"])
        assert _rel(sy["X"].cpu().numpy(), want) < TOL64
    batch.capture()
    for sy in systems:
        sy["X"].fill_(float("nan"))
    batch.launch_graph()
    batch.launch_graph()
    assert batch.status()[0] == 0
    for sy, x0 in zip(systems, first):
        assert torch.equal(sy["X"], x0)


def test_batch_result_is_the_same_alone_and_in_the_mix(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    systems = _systems(30, 500, 64, seed=4)
    g.Batch(systems).run()
    for i in (0, 7, 19):
        sy = systems[i]
        alone = dict(sy)
        alone["X"] = torch.empty_like(sy["X"].t()).t()
        b = g.Batch([alone])
        b.run()
        assert b.status()[0] == 0
        assert torch.equal(alone["X"], sy["X"])


def test_batch_reports_singular_item(cuda_lib):
    import paper_1612_01855_gb300 as g
    systems = _systems(6, 120, 8, seed=5)
    bad = systems[4]
    n = bad["Lh"].shape[0]
    r = n // 2
    bad["L"][r, r] = 0.0
    rc, item, row = (lambda b: (b.run(), b.status())[1])(g.Batch(systems))
    assert rc == -2 and item == 4 and row == r


def test_batch_argument_errors(cuda_lib):
    import paper_1612_01855_gb300 as g
    systems = _systems(2, 50, 4, seed=6)
    systems[1]["n0"] = 48  # only 32 and 64 are inverted in-launch
    with pytest.raises(g.TrsmError):
        g.Batch(systems)
    systems[1]["n0"] = 32
    systems[1]["X"] = systems[1]["B"]  # X must not alias B
    with pytest.raises(g.TrsmError):
        g.Batch(systems)


def test_batch_tile_shapes_give_identical_results(cuda_lib):
    """1- to 32-wide column tiles only change which thread computes which
    output, not the order of any sum: results are bitwise equal (tiles of 1
    to 3 columns are held by one warp, the others by all four)."""
    import torch
    import paper_1612_01855_gb300 as g
    systems = _systems(24, 400, 40, seed=8)
    ref = None
    for tile in (0, 1, 2, 3, 4, 8, 12, 16, 20, 24, 28, 32):
        for sy in systems:
            sy["tile_cols"] = tile
            sy["X"].fill_(float("nan"))
        b = g.Batch(systems)
        b.run()
        assert b.status()[0] == 0
        got = [sy["X"].clone() for sy in systems]
        if ref is None:
            ref = got
            for sy in systems:
                assert _rel(sy["X"].cpu().numpy(), oracle.forward_subst(sy["Lh"], sy["Bh"])) < TOL64
        else:
            assert all(torch.equal(a, c) for a, c in zip(ref, got)), tile
    systems[0]["tile_cols"] = 18
    with pytest.raises(g.TrsmError):
        g.Batch(systems)


def test_batch_column_split_is_bitwise_neutral(cuda_lib):
    """Items with k above 32 and not a multiple of it run as a 32-wide part
    and a narrow remainder part that shares the first part's inverted
    blocks (or the plan): the bits equal those of 32-wide tiles throughout,
    and a zero pivot is still reported by item and row."""
    import torch
    import paper_1612_01855_gb300 as g
    systems = []
    for i, (n, k) in enumerate([(150, 33), (300, 40), (97, 100), (64, 65), (500, 47), (33, 200), (120, 43),
                                (210, 52), (200, 34), (90, 67), (77, 1), (260, 2), (45, 3)]):
        L, B = inputs.well_conditioned(n, k, seed=2100 + i)
        systems.append({"Lh": L, "Bh": B, "L": _dev(L, np.float64), "B": _dev(B, np.float64),
                        "X": torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t(),
                        "n0": (32, 64)[i % 2]})
    plan = g.trsm_plan(systems[4]["L"], 100)
    systems[4]["plan"] = plan
    got = {}
    for tile in (0, 32):
        for sy in systems:
            sy["tile_cols"] = tile
            sy["X"].fill_(float("nan"))
        b = g.Batch(systems)
        b.run()
        assert b.status()[0] == 0
        got[tile] = [sy["X"].clone() for sy in systems]
    assert all(torch.equal(a, c) for a, c in zip(got[0], got[32]))
    for sy, x in zip(systems, got[0]):
        assert _rel(x.cpu().numpy(), oracle.forward_subst(sy["Lh"], sy["Bh"])) < TOL64
    for sy in systems:
        sy["tile_cols"] = 0
    systems[1]["L"][200, 200] = 0.0  # n = 300, k = 40: split into 32 + 8 columns
    b = g.Batch(systems)
    b.run()
    rc, item, row = b.status()
    assert rc == -2 and item == 1 and row == 200


def test_autotuner_choices(cuda_lib):
    from paper_1612_01855_gb300 import autotune
    table = autotune.tune_batch("f64", count=12, kmax=32, reps=1)
    assert set(table) == set(range(len(autotune.BUCKETS)))
    for n0, tile in table.values():
        assert n0 in autotune.N0_CANDIDATES and tile in autotune.TILE_CANDIDATES
    assert autotune.choose(700, "f64", table) == table[autotune.bucket_of(700)]
