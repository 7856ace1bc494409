"""Argument checks of the Python binding that run before the C library is
called (no GPU needed): gt_query_static reads and writes its tensors in
place, so a mistyped, short or non-contiguous buffer must be refused up
front."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture()
def fake_tree():
    from paper_2311_02573_gb300 import gt

    class FakeTree(gt.Tree):
        dim = 8                     # no library handle: the checks come first

        def close(self):
            pass

    t = object.__new__(FakeTree)
    t._h = None
    return t


def _args(B=4, d=8):
    return (torch.zeros(B, d), torch.full((B,), 0.9), torch.zeros(B + 1, dtype=torch.int64),
            torch.zeros(64, dtype=torch.int32))


@pytest.mark.parametrize("case, exc", [
    ("q_float64", TypeError), ("q_width", ValueError), ("q_noncontig", ValueError),
    ("q_1d", ValueError), ("rho_float64", TypeError), ("rho_short", ValueError),
    ("off_int32", TypeError), ("off_short", ValueError), ("ids_int64", TypeError),
    ("ids_noncontig", ValueError), ("host", TypeError), ("numpy", TypeError)])
def test_query_static_refuses_bad_arguments(fake_tree, case, exc):
    Q, rho, off, ids = _args()
    if case == "q_float64":
        Q = Q.double()
    elif case == "q_width":
        Q = torch.zeros(4, 7)
    elif case == "q_noncontig":
        Q = torch.zeros(8, 4).t()            # shape (4, 8), column-major
        assert not Q.is_contiguous()
    elif case == "q_1d":
        Q = torch.zeros(8)
    elif case == "rho_float64":
        rho = rho.double()
    elif case == "rho_short":
        rho = rho[:3]
    elif case == "off_int32":
        off = off.to(torch.int32)
    elif case == "off_short":
        off = off[:4]
    elif case == "ids_int64":
        ids = ids.to(torch.int64)
    elif case == "ids_noncontig":
        ids = ids[::2]
    elif case == "numpy":
        Q = Q.numpy()
    # "host": every argument is well formed but lives in host memory
    with pytest.raises(exc):
        fake_tree.query_static(Q, rho, off, ids)


def test_load_refuses_files_that_are_not_checkpoints(tmp_path):
    # checked before any device work: runs without a GPU
    from paper_2311_02573_gb300 import build, gt
    build.build()
    bad = tmp_path / "not_a_tree.gt"
    bad.write_bytes(b"this is not a tree checkpoint" * 8)
    for path in (str(bad), str(tmp_path / "missing.gt")):
        with pytest.raises(gt.GTError) as e:
            gt.Tree.load(path)
        assert e.value.status == 1
