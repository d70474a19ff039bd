"""The run-to-steady stall rule (lbc_set_stall_window), host logic on the CPU.

The rule (csrc/lbc_stall.h) sees the residual every 64 steps and stops an instance none of whose
residuals over its last `window` steps is below 0.99 times its lowest residual before them. These
tests compile it into a small driver and feed it synthetic residual histories: a geometric
contraction never stalls, however slow, as long as rate^window < 0.99; one that reaches a noise
floor stalls within about two windows of reaching it; a contraction slower than that, or a rise
that lasts a window, is (as documented) taken for a stall; nothing stalls before a full window
is sampled.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1810_07803_gb300", "csrc")
EVERY = 64   # steps per residual sample (the graph of steps)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("stall") / "stall_driver")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "stall_driver.cpp"), "-o", exe],
                   check=True)

    def run(window, residuals):
        text = f"{window}\n" + "".join(f"{EVERY * (k + 1)} {float(r)!r}\n" for k, r in enumerate(residuals))
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
        return int(out.stdout.split()[0])

    return run


def geometric(r0, rate, steps):
    return [r0 * rate ** (EVERY * (k + 1)) for k in range(steps // EVERY)]


@pytest.mark.parametrize("rate", [0.999, 0.9999, 0.999997])
def test_contraction_never_stalls(driver, rate):
    window = 4096   # rate^window = 0.017, 0.66, 0.988: each window sets a new low by more than 1 %
    assert driver(window, geometric(1e-2, rate, 400_000)) == -1


def test_noise_floor_stalls_within_a_window(driver):
    rng = np.random.default_rng(3)
    window, floor_at = 4096, 30_016
    res = geometric(1e-2, 0.9995, floor_at)            # 1e-2 -> 3e-9
    floor = res[-1]
    res += list(floor * rng.uniform(0.7, 1.3, 2000))   # wanders about the floor
    at = driver(window, res)
    assert floor_at < at <= floor_at + 2 * window, at


def test_contraction_below_one_percent_per_window_counts_as_stalled(driver):
    # rate^window = 0.9959 > 0.99: the window is the caller's bound on the slowest contraction
    at = driver(4096, geometric(1e-2, 0.999999, 100_000))
    assert at == 4096 + EVERY


def test_a_rise_lasting_a_window_counts_as_stalled(driver):
    rise = [1e-6 * 1.0005 ** (EVERY * (k + 1)) for k in range(20_000 // EVERY)]
    assert driver(4096, rise) == 4096 + EVERY


def test_nothing_stalls_before_one_window(driver):
    window = 4096
    flat = [1e-3] * 200
    at = driver(window, flat)
    assert at == window + EVERY   # the first sample with one older than the window behind it
    assert driver(window, flat[: window // EVERY]) == -1


def test_a_transient_rise_within_the_window_is_not_a_stall(driver):
    # the residual first rises for 1,000 steps (start-up), then contracts at rate 0.999
    rise = [1e-4 * 1.002 ** (EVERY * (k + 1)) for k in range(1000 // EVERY)]
    res = rise + geometric(rise[-1], 0.999, 60_000)
    assert driver(4096, res) == -1
