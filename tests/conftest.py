import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (run with -m gpu)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def synth():
    from paper_2605_23538_gb300 import synth as s
    return s


@pytest.fixture(scope="session")
def cat_c1(synth):
    return synth.catalogue("c1")


def smooth_row(n_z, z_max=2.0):
    """A smooth, positive LOS row (unit trapezoid area) for tests that integrate."""
    z = np.linspace(0.0, z_max, n_z)
    row = (0.05 + z ** 2) * np.exp(-z / 0.6)
    dz = z[1] - z[0]
    area = dz * (row.sum() - 0.5 * (row[0] + row[-1]))
    return (row / area).astype(np.float32)


def tiny_catalogue(rows, events, injections, n_draw, z_max=2.0):
    """Build a catalogue dict from explicit lists.

    rows: [n_pix, n_z]; events: list of lists of (m1d, m2d, dL, lnpi, pix);
    injections: list of (m1d, m2d, dL, lnpdraw).
    """
    rows = np.asarray(rows, dtype=np.float32)
    counts = [len(e) for e in events]
    flat = [s for e in events for s in e]
    a = np.array(flat, dtype=np.float64).reshape(-1, 5)
    inj = np.array(injections, dtype=np.float64).reshape(-1, 4)
    return dict(offsets=np.concatenate([[0], np.cumsum(counts)]).astype(np.int64),
                m1=a[:, 0].astype(np.float32), m2=a[:, 1].astype(np.float32),
                dl=a[:, 2].astype(np.float32), lnpe=a[:, 3].astype(np.float32),
                pix=a[:, 4].astype(np.int32), los=rows, z_max=float(z_max),
                inj_m1=inj[:, 0].astype(np.float32), inj_m2=inj[:, 1].astype(np.float32),
                inj_dl=inj[:, 2].astype(np.float32), inj_lnpd=inj[:, 3].astype(np.float32),
                n_draw=float(n_draw))


# Grid positions closer than this (in cells) to a node: the library's FP32 position,
# accurate to ~1e-7 of a cell, may put such a sample on either side of the node, and the
# two cells then give the same interpolated value (the prior is continuous there).
NODE_WINDOW = 2e-5


def cell_mismatches(got, ref_cell, ref_pos):
    """Compare the library's per-sample LOS cells with the oracle's (cell and exact grid
    position from oracle.sample_cells).  Returns (n_checked, n_near, n_diff_near); raises
    AssertionError for any difference away from a node, or a difference near a node other
    than the neighbouring cell."""
    got = np.asarray(got)
    assert np.array_equal(got >= 0, ref_cell >= 0), "samples inside / outside [0, z_max] differ"
    inside = ref_cell >= 0
    pos = ref_pos[inside]
    near = np.abs(pos - np.round(pos)) < NODE_WINDOW
    g, r = got[inside], ref_cell[inside]
    far_bad = (g != r) & ~near
    assert not far_bad.any(), (f"{far_bad.sum()} cells differ away from any node, e.g. position "
                               f"{pos[far_bad][:3]}, library {g[far_bad][:3]}, oracle {r[far_bad][:3]}")
    node = np.round(pos[near]).astype(np.int64)
    gn = g[near]
    ok_near = (gn == node) | (gn == node - 1)
    assert ok_near.all(), "a cell near a node is neither of the node's two cells"
    return int(inside.sum()), int(near.sum()), int((g[near] != r[near]).sum())
