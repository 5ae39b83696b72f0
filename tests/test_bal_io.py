"""Bundle-Adjustment-in-the-Large text files (mba_bal_read / mba_bal_write), the
graph-style problem declaration (mba.Graph) and the batched windows' array
assembly (mba.concat_windows).  Host only, except
test_graph_problem_solves_like_the_arrays, which solves on the GPU."""
import numpy as np
import pytest

from scenes import make_scene


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


def _arrays(sc):
    return sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx


def test_round_trip_is_bit_exact(mba, tmp_path):
    sc = make_scene(7, 300, sigma=0.5, seed=3)
    path = tmp_path / "scene.txt"
    mba.mba_bal_write(path, *_arrays(sc))
    got = mba.mba_bal_read(path)
    for a, b in zip(got, _arrays(sc)):
        np.testing.assert_array_equal(a, np.asarray(b).reshape(a.shape))
        assert a.dtype == np.asarray(b).dtype


def test_reads_the_documented_layout(mba, tmp_path):
    # 2 cameras, 3 points, 4 observations, whitespace of several kinds
    text = """2 3 4
0 0 -1.5e+01 2.25
1 0 3.0 -4.0
0 2   0.5\t0.25
1 1 10 -10
0.1
-0.2
0.3
0
0
-5
800
0.01
-0.001
0
0
0
1
2
-6
900
0
0
0.5 -0.5 0.25
1 1 1
-1 0 2
"""
    path = tmp_path / "tiny.txt"
    path.write_text(text)
    cams, pts, obs, ci, pi = mba.mba_bal_read(path)
    np.testing.assert_array_equal(ci, [0, 1, 0, 1])
    np.testing.assert_array_equal(pi, [0, 0, 2, 1])
    np.testing.assert_array_equal(obs, [[-15.0, 2.25], [3.0, -4.0], [0.5, 0.25], [10.0, -10.0]])
    np.testing.assert_array_equal(cams, [[0.1, -0.2, 0.3, 0, 0, -5, 800, 0.01, -0.001],
                                         [0, 0, 0, 1, 2, -6, 900, 0, 0]])
    np.testing.assert_array_equal(pts, [[0.5, -0.5, 0.25], [1, 1, 1], [-1, 0, 2]])


@pytest.mark.parametrize("text,status", [
    ("", "INVALID_ARG"),                                       # no header
    ("1 1 0\n", "INVALID_ARG"),                                # n < 1
    ("1 1 1\n0 0 1.0\n", "INVALID_ARG"),                       # truncated observation
    ("1 1 1\n0 1 1 2\n" + "0\n" * 9 + "0 0 0\n", "INVALID_ARG"),  # point index out of range
    ("1 1 1\n0 0 1 2\n" + "0\n" * 8, "INVALID_ARG"),           # truncated camera block
    ("1 1 1\n0 0 1 2\n" + "0\n" * 9 + "0 0\n", "INVALID_ARG"),   # truncated point
    ("1 1 1\n0 0 nan 2\n" + "0\n" * 9 + "0 0 0\n", "NONFINITE"),
])
def test_malformed_files_are_rejected(mba, tmp_path, text, status):
    path = tmp_path / "bad.txt"
    path.write_text(text)
    with pytest.raises(mba.MbaError, match=status):
        mba.mba_bal_read(path)


@pytest.mark.parametrize("suffix", [".bz2", ".gz", ".xz"])
def test_compressed_files_round_trip(mba, tmp_path, suffix):
    """The BAL datasets ship bz2-compressed: a compressed path is written
    through, and read back from, the standard-library codec of its suffix."""
    import bz2
    import gzip
    import lzma

    codec = {".bz2": bz2, ".gz": gzip, ".xz": lzma}[suffix]
    sc = make_scene(4, 120, sigma=0.5, seed=6)
    path = tmp_path / ("scene.txt" + suffix)
    mba.mba_bal_write(path, *_arrays(sc))
    with codec.open(path, "rt") as f:  # really compressed, and the header is the BAL one
        assert f.readline().split() == [str(sc.nc), str(sc.np_), str(sc.n)]
    got = mba.mba_bal_read(path)
    for a, b in zip(got, _arrays(sc)):
        np.testing.assert_array_equal(a, np.asarray(b).reshape(a.shape))
    plain = tmp_path / "plain.txt"
    mba.mba_bal_write(plain, *_arrays(sc))
    assert codec.decompress(path.read_bytes()) == plain.read_bytes()


def test_missing_file_is_rejected(mba, tmp_path):
    with pytest.raises(mba.MbaError, match="INVALID_ARG"):
        mba.mba_bal_read(tmp_path / "absent.txt")


def test_graph_declaration_matches_the_arrays(mba, tmp_path):
    sc = make_scene(5, 80, sigma=0.5, seed=4)
    g = mba.Graph()
    cam_ids = [g.add_camera(c) for c in sc.cameras]
    pt_ids = [g.add_point(p) for p in sc.points]
    for k in range(sc.n):
        g.add_edge(cam_ids[sc.cam_idx[k]], pt_ids[sc.pt_idx[k]], sc.observations[k])
    for a, b in zip(g.arrays(), _arrays(sc)):
        np.testing.assert_array_equal(a, np.asarray(b).reshape(a.shape))
    with pytest.raises(IndexError):
        g.add_edge(len(cam_ids), 0, (0.0, 0.0))
    path = tmp_path / "graph.txt"
    g.to_bal(path)
    for a, b in zip(mba.Graph.from_bal(path).arrays(), g.arrays()):
        np.testing.assert_array_equal(a, b)


@pytest.mark.gpu
def test_graph_problem_solves_like_the_arrays(mba, tmp_path):
    sc = make_scene(8, 400, sigma=0.5, seed=5)
    path = tmp_path / "scene.txt"
    mba.mba_bal_write(path, *_arrays(sc))
    opts = dict(max_iter=6, pcg_max_iter=40)
    with mba.Graph.from_bal(path).problem() as pr:
        s1 = pr.solve(**opts)
        c1, p1 = pr.parameters()
    with mba.Problem(*_arrays(sc)) as pr:
        s2 = pr.solve(**opts)
        c2, p2 = pr.parameters()
    assert s1["final_cost"] == s2["final_cost"]
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(p1, p2)


def test_concat_windows_keeps_window_local_indices(mba):
    """Batched windows are passed as concatenated arrays plus per-window
    offsets; indices stay local to their window (host logic, no GPU)."""
    ws = [make_scene(nc, npt, sigma=0.5, seed=40 + nc) for nc, npt in ((5, 30), (7, 44), (6, 25))]
    co, po, oo, cams, pts, obs, ci, pi = mba.concat_windows(
        [(s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx) for s in ws])
    assert co.tolist() == [0, 5, 12, 18] and po.tolist() == [0, 30, 74, 99]
    assert oo.tolist() == np.cumsum([0] + [s.n for s in ws]).tolist()
    assert co.dtype == po.dtype == oo.dtype == np.int64 and ci.dtype == pi.dtype == np.int32
    for w, s in enumerate(ws):
        np.testing.assert_array_equal(cams[co[w]:co[w + 1]], s.cameras)
        np.testing.assert_array_equal(pts[po[w]:po[w + 1]], s.points)
        np.testing.assert_array_equal(obs[oo[w]:oo[w + 1]], s.observations)
        np.testing.assert_array_equal(ci[oo[w]:oo[w + 1]], s.cam_idx)
        np.testing.assert_array_equal(pi[oo[w]:oo[w + 1]], s.pt_idx)
