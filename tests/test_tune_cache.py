"""The autotuner's cache file (host only, no GPU): a saved cache loads back to the same
file, a malformed entry or header is rejected with ZKVC_EIO and changes nothing."""
import pytest

from tests import _util


@pytest.fixture(scope="module")
def nv():
    return _util.native()


GOOD = ("zkvc-tune-cache 1\n"
        "49 320 512 2 152 0 0 16 8 10 0 1 1 0 0 NVIDIA_GB300\n"
        "4 16 8 1 152 2 4 8 16 9 2 1 0 1 1 NVIDIA_GB300\n")


def test_cache_round_trip(nv, tmp_path):
    nv.zkvc_tune_cache_clear()
    src = tmp_path / "a.txt"
    src.write_text(GOOD)
    nv.zkvc_tune_cache_load(src)
    out = tmp_path / "b.txt"
    nv.zkvc_tune_cache_save(out)
    assert sorted(out.read_text().splitlines()) == sorted(GOOD.splitlines())
    nv.zkvc_tune_cache_clear()
    nv.zkvc_tune_cache_save(out)
    assert out.read_text() == "zkvc-tune-cache 1\n"


@pytest.mark.parametrize("bad", [
    "not a cache\n",
    "zkvc-tune-cache 1\n49 320 512 2 152 0 0 16 8 12 0 1 1 0 0 X\n",      # NTT block 2^12
    "zkvc-tune-cache 1\n49 320 512 2 152 0 0 16 8 10 3 1 1 0 0 X\n",      # side start 3
    "zkvc-tune-cache 1\n49 320 512 7 152 0 0 16 8 10 0 1 1 0 0 X\n",      # mode 7
    "zkvc-tune-cache 1\n49 320 512 2 152 0 0 16\n",                       # short line
    "zkvc-tune-cache 1\n0 320 512 2 152 0 0 16 8 10 0 1 1 0 0 X\n",       # a = 0
])
def test_cache_rejects_malformed(nv, tmp_path, bad):
    nv.zkvc_tune_cache_clear()
    good = tmp_path / "g.txt"
    good.write_text(GOOD)
    nv.zkvc_tune_cache_load(good)
    p = tmp_path / "bad.txt"
    p.write_text(bad)
    with pytest.raises(nv.ZkvcError) as e:
        nv.zkvc_tune_cache_load(p)
    assert e.value.code == nv.ZKVC_EIO
    out = tmp_path / "o.txt"
    nv.zkvc_tune_cache_save(out)
    assert sorted(out.read_text().splitlines()) == sorted(GOOD.splitlines())
    with pytest.raises(nv.ZkvcError):
        nv.zkvc_tune_cache_load(tmp_path / "missing.txt")
