"""Strip groups (Divide & Recombine with bounded memory, Sect. 4.1's
carryover buffers): a single series whose boundary descriptors exceed the
budget runs G strips at a time, and the open run of every row and diagonal
crossing a group's left edge is carried to the next group.  Budgets forced
down to a few hundred kilobytes (RQA_DESC_BUDGET) give dozens of groups on
series the materialised or streaming oracle checks exactly: every norm,
Theiler windows, strip widths, groups of one strip, and constant and
periodic series whose lines cross every group."""
import numpy as np
import pytest

import synth
from gpu_util import check_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _no_bands(monkeypatch):
    monkeypatch.setenv("RQA_BAND_ROWS", "0")   # groups apply to unbanded strips
    monkeypatch.delenv("RQA_TILE_WARPS", raising=False)
    monkeypatch.delenv("RQA_TILE_COLS", raising=False)


@pytest.mark.parametrize("budget", [40_000, 150_000, 400_000])
@pytest.mark.parametrize("norm", [0, 1, 2])
def test_groups_exact(monkeypatch, budget, norm):
    monkeypatch.setenv("RQA_DESC_BUDGET", str(budget))
    monkeypatch.setenv("RQA_TILE_WARPS", "2")
    monkeypatch.setenv("RQA_TILE_COLS", "4")
    s = synth.ar1(6000, 500 + norm, 0.93)
    r, st, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=norm, theiler=1)
    assert st["strip_groups"] > 1
    assert st["strip_groups"] * st["strips_per_group"] * st["strip_width"] >= st["n_vec"] - 1


@pytest.mark.parametrize("warps", [1, 2, 8])
@pytest.mark.parametrize("w", [0, 3, 700])
def test_groups_widths_windows(monkeypatch, warps, w):
    monkeypatch.setenv("RQA_DESC_BUDGET", "20000")
    monkeypatch.setenv("RQA_TILE_WARPS", str(warps))
    s = synth.lorenz_x(4000, 600 + warps + w, discard=1500)
    r, st, _ = check_parity(s, m=4, tau=2, eps=0.6, norm=0, theiler=w)
    assert st["strip_groups"] > 1


def test_one_strip_per_group_and_long_lines(monkeypatch):
    """A budget below one strip's descriptors: every group is one strip.
    Constant and periodic series put black runs across every group's edge
    (diagonals of full length, rows of up to n cells)."""
    monkeypatch.setenv("RQA_DESC_BUDGET", "1")
    monkeypatch.setenv("RQA_TILE_WARPS", "1")
    for s in (synth.constant(3000), synth.periodic(3000, 7)):
        for w in (0, 1):
            r, st, _ = check_parity(s, m=2, tau=1, eps=0.5, norm=1, theiler=w)
            assert st["strips_per_group"] == 1 and st["strip_groups"] > 20


def test_groups_are_not_used_below_the_budget(monkeypatch):
    monkeypatch.setenv("RQA_DESC_BUDGET", str(1 << 30))
    s = synth.ar1(6000, 77, 0.93)
    r, st, _ = check_parity(s, m=3, tau=1, eps=0.5, norm=1, theiler=1)
    assert st["strip_groups"] == 1 and st["desc_bytes"] == st["desc_bytes_all_strips"]
