"""Sec. 4.1 wavespeed recovery (E1) with the oracle, on the paper's setup read
from tests/golden/wavespeed_e1.json: 180^3 nodes at dx = 0.2 mm, rho = 1000,
c_s = 2 m/s, eta = 0, a curl source, u_z traces at 3.6, 6.0, 8.4 and 10.8 mm
along x, peak-arrival times refined by a parabola and a least-squares
distance-time fit.

The paper reports 1.998 m/s (< 0.1 %) but not its source width, and states
(Sec. 4.2) that the peak-picked speed carries a source-width- and
near-field-dependent bias. With the curl of a Gaussian envelope in the x-y
plane the oracle gives 1.989 m/s for a 1 mm envelope and 2.067 m/s for 3 mm
(2.16 m/s for a 3 mm envelope in all three axes): the sensors sit 1.2 to 3.6
widths from a 3 mm source, in its near field. So the 0.1 % figure is not a
pin of this implementation; the narrow-source run is gated at 1 % and the
wavespeed itself is pinned at 0.1 % by the 1D Kelvin-Voigt chain at eta = 0
(tests/test_oracle_kv_benchmark.py).
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_2607_28414_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
E1 = json.load(open(os.path.join(HERE, "golden", "wavespeed_e1.json")))


def test_e1_sensors_fall_on_nodes():
    dx = E1["dx_m"]
    cells = [o / dx for o in E1["sensor_offsets_m"]]
    assert np.allclose(cells, np.round(cells), atol=1e-9)
    assert [int(round(c)) for c in cells] == [18, 30, 42, 54]
    assert E1["grid"][0] * dx == pytest.approx(0.036)


@pytest.mark.slow
def test_e1_linear_fit_wavespeed_narrow_source():
    n = E1["grid"][0]
    dx = E1["dx_m"]
    rho, cs = E1["rho"], E1["c_s"]
    G = rho * cs ** 2
    v0 = inputs.curl_gaussian_velocity(n, n, n, dx, sigma=1e-3, envelope="xy")
    c = n // 2
    offs = E1["sensor_offsets_m"]
    sens = np.array([[c + int(round(o / dx)), c, c] for o in offs], np.int32)
    dt = 0.5 * orc.stable_dt(G, rho, 0.0, dx)
    n_steps = int(8e-3 / dt) + 2
    tr = orc.run(n, n, n, dx, dt, G, rho, 0.0, n_steps, sens, v0=v0)
    ttp = [orc.time_to_peak(tr[:, s, 2], dt) for s in range(len(offs))]
    fit = orc.linear_fit_speed(offs, ttp)
    mean = float(np.mean(np.array(offs) / np.array(ttp)))
    print(f"E1 (1 mm source): linear fit {fit:.4f} m/s, mean TTP speed {mean:.4f} m/s "
          f"(paper: {E1['linear_fit_speed_m_s']} and {E1['mean_ttp_speed_m_s']} with its source)")
    assert abs(fit - cs) <= 0.01 * cs
