"""Model-file reader (the command language of the paper's command-line
program, Sec. 3 and the model files of Sec. 4): a model file must build the
scenario it describes, and that scenario must run exactly like one built by
hand (FP64 oracle, CPU only)."""
import math

import numpy as np
import pytest

from _scenario import oracle_from_scenario
from paper_2207_06908_gb300 import modelfile as M
from paper_2207_06908_gb300 import workloads as W

MODEL = """
# a buried rod with a riser, an inclined arm from the riser's top, a gap source
volume (3.0, 2.5, 2.0, 0.1)            # 30 x 25 x 20 cells
calctime (2e-8)
output (1e-9)
abc (cpml, 0.4, 1, 1, 1e-3, 3, 1)
block (0, 0, 0, 3.0, 2.5, 1.0, 10, 0.01, soil)
block (1.0, 1.0, 0.5, 2.0, 2.0, 1.0, 4, 0.001)
debye (soil, 20, 1e-8, 5, 1e-9)
wire (thin, 1.5, 1.2, 0.6, 1.5, 1.2, 1.3, 0.004)
wire (thin, 1.5, 1.2, 1.3, 2.05, 1.52, 1.47, 0.003, t)
source (current, 1.5, 1.2, 1.3, 1.5, 1.2, 1.4, 0, fn)
calculate (current, 1.5, 1.2, 0.9, 1.5, 1.2, 0.8)
calculate (voltage, 1.5, 1.3, 1.3, 1.5, 1.6, 1.3)
function (fn, ramp, 100, 5e-9)
"""


def by_hand(courant):
    n, dx = (30, 25, 20), 0.1
    cm = W.paint_blocks(n, [((0, 0, 0), (30, 25, 10), 1), ((10, 10, 5), (20, 20, 10), 2)])
    steps = math.ceil(2e-8 / W.time_step(dx, courant))
    cur = W.ramp(W.sample_times(steps, dx, courant), 100.0, 5e-9)
    sc = W.Scenario("hand", n, dx, courant, 4, cm, [(1.0, 0.0, 1.0), (10.0, 0.01, 1.0), (4.0, 0.001, 1.0)],
                    wires=[((15, 12, 6), (15, 12, 13), 0.004)], sources=[((15, 12, 13), 2, cur)],
                    probes=[(W.PROBE_I, (15, 12, 8), 2, 1), (W.PROBE_V, (15, 13, 13), 1, 3)], n_steps=steps)
    sc.debye = {1: ([20.0, 5.0], [1e-8, 1e-9])}
    sc.owires = [((15.0, 12.0, 13.0), (20.5, 15.2, 14.7), 0.003)]
    return sc


def test_reads_a_model_into_the_scenario_it_describes():
    m = M.parse(MODEL, courant=0.9)
    sc, ref = m.scenario, by_hand(0.9)
    assert sc.n == ref.n and sc.dx == ref.dx and sc.cpml == 4 and sc.n_steps == ref.n_steps == 116
    assert sc.materials == ref.materials and sc.debye == ref.debye
    assert np.array_equal(sc.cell_material, ref.cell_material)
    assert sc.wires == ref.wires
    assert sc.owires == ref.owires
    assert [s[:2] for s in sc.sources] == [s[:2] for s in ref.sources]
    assert np.array_equal(sc.sources[0][2], ref.sources[0][2])
    assert sc.probes == ref.probes
    assert m.output_dt == 1e-9
    assert [(k, s) for k, _, s in m.probe_names] == [("current", -1), ("voltage", 1)]


def test_parsed_model_runs_exactly_like_the_hand_built_one():
    sc, ref = M.parse(MODEL, courant=0.9).scenario, by_hand(0.9)
    a, b = oracle_from_scenario(sc, parity=True), oracle_from_scenario(ref, parity=True)
    a.step(60)
    b.step(60)
    for c in range(6):
        assert np.array_equal(a.get_field(c), b.get_field(c))
    for p in range(2):
        assert np.array_equal(a.read_probe(p), b.read_probe(p))
    assert float(np.abs(a.read_probe(1)).max()) > 0


def test_functions():
    t = np.linspace(0.0, 2e-6, 401)
    custom = M._waveform(["custom", "1e-7", "0", "2", "1"], t, 1)
    assert custom[0] == 0.0 and abs(np.interp(0.5e-7, t, custom) - 1.0) < 1e-9
    assert np.all(custom[t > 2e-7 + 1e-12] == 0.0)
    # Heidler without eta: the peak-corrected class function of the workloads
    h = M._waveform(["heidler", "s", "3.7e-7", "1.4e-5", "2", "10"], t, 1)
    assert np.allclose(h, W.heidler(t, 2.0, 3.7e-7, 1.4e-5, 10))
    # with eta and a delay: shifted, scaled by 1 / eta
    hd = M._waveform(["heidler", "s", "3.7e-7", "1.4e-5", "1", "10", "1", "1.85e-7"], t, 1)
    s = np.clip((t - 1.85e-7) / 3.7e-7, 0, None) ** 10
    ref = np.where(t > 1.85e-7, s / (1 + s) * np.exp(-np.clip(t - 1.85e-7, 0, None) / 1.4e-5), 0.0)
    assert np.allclose(hd, ref)
    d = M._waveform(["dexp", "5", "1e4", "1e6"], t, 1)
    assert np.allclose(d, 5 * (np.exp(-1e4 * t) - np.exp(-1e6 * t)))


def test_resample_to_the_output_interval():
    m = M.parse(MODEL, courant=0.9)
    dt = W.time_step(0.1, 0.9)
    x = np.arange(m.scenario.n_steps, dtype=float)
    t, v = m.resample(x, "current")
    assert abs(t[1] - 1e-9) < 1e-21 and np.allclose(v, np.interp(t, (x + 0.5) * dt, x, left=0.0))
    t, v = m.resample(x, "voltage")
    assert np.allclose(v, np.interp(t, (x + 1.0) * dt, x, left=0.0))


@pytest.mark.parametrize("bad, where", [
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\nfoo (1)\n", "line 3"),
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\nblock (0, 0, 0, 1, 1)\n", "line 3"),
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\nsource (current, 0.5, 0.5, 0.5, 0.5, 0.5, 0.7, 0, f)\n"
     "function (f, ramp, 1, 1e-9)\n", "line 3"),
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\nsource (current, 0.5, 0.5, 0.5, 0.5, 0.5, 0.6, 0, g)\n", "line 3"),
    ("calctime (1e-9)\n", "volume"),
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\ncalculate (voltage, 0.5, 0.5, 0.5, 0.6, 0.6, 0.5)\n", "line 3"),
    ("volume (1, 1, 1, 0.1)\ncalctime (1e-9)\nwire (thin, 0.55, 0.5, 0.5, 0.55, 0.5, 0.7, 0.001)\n"
     "wire (bent, 0, 0, 0, 1, 1, 1, 0.001)\n", "line 4"),
])
def test_errors_name_the_line(bad, where):
    with pytest.raises(ValueError, match=where):
        M.parse(bad)


def test_cli_parse_only(tmp_path, capsys):
    p = tmp_path / "model.txt"
    p.write_text(MODEL)
    assert M.main([str(p), "--parse-only", "--courant", "0.9"]) == 0
    out = capsys.readouterr().out
    assert "30x25x20 cells" in out and "1 thin + 1 oblique" in out and "2 probes" in out


def test_probe_orientation_follows_the_file():
    """the same current probe and voltage path written in both directions
    read, after the model's sign, exact opposites: each measures from its
    first point to its second (oracle run)"""
    text = MODEL + """
calculate (current, 1.5, 1.2, 0.8, 1.5, 1.2, 0.9)
calculate (voltage, 1.5, 1.6, 1.3, 1.5, 1.3, 1.3)
"""
    m = M.parse(text, courant=0.9)
    assert [s for _, _, s in m.probe_names] == [-1, 1, 1, -1]
    o = oracle_from_scenario(m.scenario, parity=True)
    o.step(80)
    p = [s * o.read_probe(q) for q, (_, _, s) in enumerate(m.probe_names)]
    assert np.array_equal(p[0], -p[2]) and np.array_equal(p[1], -p[3])
    assert float(np.abs(p[1]).max()) > 0 and float(np.abs(p[0]).max()) > 0
