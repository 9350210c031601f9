"""Angular discretisation study of Sec. VI-A on the GPU path: against a fine
Dirac (pinhole) rendering, both bases converge as the lens grid is refined,
the pillbox basis is the more accurate one at coarse grids, and it costs about
the same time as the Dirac basis at equal K."""
import pytest

torch = pytest.importorskip("torch")

from paper_1812_03358_b300 import build

pytestmark = pytest.mark.gpu


def test_pillbox_beats_dirac_at_coarse_grids_at_equal_cost():
    build.build()
    from paper_1812_03358_b300 import accuracy as A
    res = A.angular_study(grid=(2, 4, 8), ref=32, n_vox=48, n_lenslets=24)
    rows = {(r["basis"], r["grid"]): r for r in res["rows"]}
    assert all("nsd" in r for r in rows.values()), res
    for basis in ("pillbox", "dirac"):
        nsds = [rows[(basis, g)]["nsd"] for g in (2, 4, 8)]
        assert nsds[0] > nsds[1] > nsds[2], (basis, nsds)
    for g in (2, 4):
        assert rows[("pillbox", g)]["nsd"] < rows[("dirac", g)]["nsd"], res
    for g in (4, 8):
        ratio = rows[("pillbox", g)]["forward_ms"] / rows[("dirac", g)]["forward_ms"]
        assert 0.5 < ratio < 2.0, (g, ratio)
