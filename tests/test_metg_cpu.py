"""Task Bench's METG(50) computation (bench.metg50) on synthetic efficiency
curves whose crossing is known in closed form."""
import numpy as np

import bench


def curve(overhead_ms, steps, ns_per_iter, iters):
    """Runs whose time is a fixed overhead plus steps x iters x the body's time:
    efficiency = useful / (overhead + useful), which is 1/2 where the useful time
    equals the overhead, i.e. at granularity 2 x overhead / steps."""
    walls = [overhead_ms + steps * it * ns_per_iter * 1e-6 for it in iters]
    eff = [steps * it * ns_per_iter * 1e-6 / w for it, w in zip(iters, walls)]
    gran = [1e3 * w / steps for w in walls]
    return gran, eff


def test_crossing_on_a_sample_is_exact():
    steps, c = 1000, 2.0
    # the useful time equals the overhead at iters = 512 exactly
    overhead = steps * 512 * c * 1e-6
    gran, eff = curve(overhead, steps, c, [0, 64, 256, 512, 2048, 8192])
    assert abs(eff[3] - 0.5) < 1e-12
    assert abs(bench.metg50(gran, eff) - 2e3 * overhead / steps) < 1e-9


def test_crossing_between_samples_is_close():
    steps, c = 1000, 1.7
    for overhead in (0.5, 2.0, 7.3, 31.0):
        iters = [0] + [int(round(16 * 1.25 ** k)) for k in range(60)]
        gran, eff = curve(overhead, steps, c, iters)
        want = 2e3 * overhead / steps
        got = bench.metg50(gran, eff)
        assert abs(got - want) / want < 0.02, (overhead, got, want)


def test_coarse_grid_stays_within_its_bracket():
    steps, c = 1000, 2.3
    iters = [0, 16, 64, 256, 1024, 4096, 16384, 65536]
    gran, eff = curve(3.0, steps, c, iters)
    got = bench.metg50(gran, eff)
    k = next(i for i, e in enumerate(eff) if e >= 0.5)
    assert gran[k - 1] <= got <= gran[k]
    want = 2e3 * 3.0 / steps
    assert abs(got - want) / want < 0.35


def test_never_and_already_efficient():
    assert bench.metg50([1.0, 2.0, 4.0], [0.1, 0.2, 0.3]) is None
    assert bench.metg50([1.0, 2.0], [0.6, 0.9]) == 1.0
    assert bench.metg50([], []) is None
    # monotone in the overhead: more overhead, larger METG
    steps, c, iters = 1000, 2.0, [0] + [2 ** k for k in range(4, 18)]
    vals = [bench.metg50(*curve(o, steps, c, iters)) for o in (1.0, 2.0, 4.0, 8.0)]
    assert all(a < b for a, b in zip(vals, vals[1:]))
    assert np.isfinite(vals).all()
