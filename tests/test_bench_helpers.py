"""Host-side helpers of bench.py (no GPU): the kinetic energy spectrum of the
double shear layer study, the assembly of a uniform grid from exported blocks,
the error against a fine reference and the clock summary of the timed region."""
import numpy as np

import bench


def test_spectrum_of_single_modes_and_parseval():
    # cos(2 pi 3 x) in psi_x and sin(2 pi 4 x) in psi_y: all energy in shells 3
    # and 4, 1/4 each (mean of cos^2 / 2), and the shells sum to the mean
    # kinetic energy density
    N = 64
    x = np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    px, py = np.cos(2 * np.pi * 3 * X), np.sin(2 * np.pi * (4 * Y))
    s = bench.kinetic_energy_spectrum(px, py, 8.0)
    assert np.allclose(s[[3, 4]], 0.25, rtol=1e-13, atol=0) and np.allclose(np.delete(s, [3, 4]), 0.0, rtol=0, atol=1e-14)
    rng = np.random.default_rng(0)
    px, py = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    s = bench.kinetic_energy_spectrum(px, py, 8.0)
    # shells beyond N/2 (the corners of the square) are cut off
    k1 = np.fft.fftfreq(N, 1.0 / N)
    inside = np.rint(np.sqrt(k1[None, :] ** 2 + k1[:, None] ** 2)) <= N // 2
    e = 0.5 * (np.abs(np.fft.fft2(px)) ** 2 + np.abs(np.fft.fft2(py)) ** 2) / N ** 4
    assert np.isclose(s.sum(), e[inside].sum(), rtol=1e-12, atol=0)


def test_uniform_field_places_blocks():
    Bs, J = 5, 2
    n = 1 << J
    info = np.zeros(n * n, dtype=[("coords", np.int32, 3)])
    f = np.zeros((n * n, 1, Bs, Bs))
    for q in range(n * n):
        cx, cy = q % n, q // n
        info["coords"][q] = (cx, cy, 0)
        i = cx * (Bs - 1) + np.arange(Bs)
        j = cy * (Bs - 1) + np.arange(Bs)
        f[q, 0] = 1000 * j[:, None] + i[None, :]
    u = bench.uniform_field(info, f, Bs, J)
    N = (Bs - 1) * n
    assert np.array_equal(u[0], 1000 * np.arange(N)[:, None] + np.arange(N)[None, :])


def test_error_vs_reference_on_adaptive_blocks():
    # blocks of levels 1 and 2 sampled from the function the reference (level
    # 3) is sampled from: zero error; a perturbation of one node of known size
    # gives the Linf error exactly
    Bs, jref = 5, 3
    Nr = (Bs - 1) << jref
    F = lambda x, y: 2.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    x = np.arange(Nr) / Nr
    ref = F(x[None, :], x[:, None])
    leaves = [(1, (0, 0))] + [(2, (cx, cy)) for cx in range(4) for cy in range(4) if cx >= 2 or cy >= 2]
    info = np.zeros(len(leaves), dtype=[("level", np.int32), ("coords", np.int32, 3)])
    f = np.zeros((len(leaves), Bs, Bs))
    for q, (lv, (cx, cy)) in enumerate(leaves):
        info["level"][q] = lv
        info["coords"][q] = (cx, cy, 0)
        xs = (cx * (Bs - 1) + np.arange(Bs)) / ((Bs - 1) << lv)
        ys = (cy * (Bs - 1) + np.arange(Bs)) / ((Bs - 1) << lv)
        f[q] = F(xs[None, :], ys[:, None])
    l2, linf = bench.error_vs_reference(info, f, ref, Bs, jref)
    assert l2 < 1e-15 and linf < 1e-15
    f[0, 1, 2] += 0.5
    l2, linf = bench.error_vs_reference(info, f, ref, Bs, jref)
    assert np.isclose(linf, 0.5 / np.abs(ref).max()) and l2 > 0


def test_clock_summary_median_and_reasons():
    # nvidia-smi csv rows (index, clocks.sm, clocks.max.sm, power, active mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap); malformed rows are skipped
    c = bench.Clocks(0)
    c.lines = ["0, 1980, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, 2070, 2070, 1000.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2010, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, [N/A], 2070",
               "garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2070, 700.0, 0x0000000000000048, Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    c.lines = []
    assert c.summary() is None
