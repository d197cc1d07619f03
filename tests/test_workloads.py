"""Host-side checks of the seeded input generators (CPU)."""
import math

import numpy as np

from paper_2207_06908_gb300 import workloads as W


def test_double_exponential_front_and_tail():
    """1.2/50 us: front time 1.25 (t90 - t10) = 1.2 us, half value at 50 us,
    peak normalised to 1 (the standard lightning-impulse shape)."""
    a, b, k = W.double_exponential_params(1.2e-6, 50e-6)
    t = np.linspace(0, 120e-6, 2_400_001)
    i = W.double_exponential(t, 1.0, a, b, k)
    p = int(np.argmax(i))
    assert abs(i[p] - 1.0) < 1e-6
    t10 = t[np.argmax(i >= 0.1)]
    t90 = t[np.argmax(i >= 0.9)]
    th = t[p + np.argmax(i[p:] <= 0.5)]
    assert abs(1.25 * (t90 - t10) - 1.2e-6) < 2e-9
    assert abs(th - 50e-6) < 1e-7


def test_config_shapes_and_steps():
    c1 = W.config1()
    assert c1.n == (48, 48, 48) and c1.n_steps == 500 and c1.cpml == 0
    assert c1.cell_material[:24].min() == 1 and c1.cell_material[24:].max() == 0
    c2 = W.config2(n_steps=8)
    assert c2.n == (256, 256, 256) and c2.cpml == 10
    assert c2.wires[0][0] == (128, 128, 129) and c2.wires[0][1] == (128, 128, 189)
    assert len(c2.probes) == 6
    dt = W.time_step(0.5, 0.99)
    assert math.isclose(dt, 0.99 * 0.5 / (W.C0 * math.sqrt(3)), rel_tol=1e-15)


def test_random_scenario_is_seeded():
    a = W.random_scenario(3)
    b = W.random_scenario(3)
    assert np.array_equal(a.cell_material, b.cell_material)
    assert all(np.array_equal(x, y) for x, y in zip(a.fields, b.fields))
    c = W.random_scenario(4)
    assert not np.array_equal(a.fields[0], c.fields[0])
