"""The surrogate's checkpoint file (sop_surrogate_file_write / _read, the
format of sop_surrogate_save / _load) on the host, without a GPU: a round
trip keeps every bit and the step, and damaged or mismatched files are
refused with a message."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def test_round_trip_is_bit_exact(sop, tmp_path):
    rng = np.random.default_rng(0)
    n = int(sop.load().sop_surrogate_param_count())
    p, m, v = (rng.standard_normal(n).astype(np.float32) for _ in range(3))
    p[0], m[1], v[2] = np.float32(-0.0), np.float32(1e-45), np.float32(3.4e38)
    f = tmp_path / "net.ckpt"
    sop.surrogate_file_write(f, 1234, p, m, v)
    raw = f.read_bytes()
    assert raw[:8] == b"SOPSURR2" and len(raw) == 16 + 12 * n
    assert int.from_bytes(raw[8:12], "little") == n and int.from_bytes(raw[12:16], "little") == 1234
    step, p2, m2, v2 = sop.surrogate_file_read(f, n)
    assert step == 1234
    for a, b in ((p, p2), (m, m2), (v, v2)):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_damaged_files_are_refused(sop, tmp_path):
    n = int(sop.load().sop_surrogate_param_count())
    z = np.zeros(n, np.float32)
    good = tmp_path / "good.ckpt"
    sop.surrogate_file_write(good, 7, z, z, z)
    raw = good.read_bytes()
    cases = {"magic": b"XOPSURR2" + raw[8:], "short": raw[:-4], "long": raw + b"\0",
             "count": raw[:8] + (n + 1).to_bytes(4, "little") + raw[12:]}
    for name, data in cases.items():
        f = tmp_path / f"{name}.ckpt"
        f.write_bytes(data)
        with pytest.raises(sop.SopError) as ei:
            sop.surrogate_file_read(f, n)
        assert ei.value.status == 1, name
    with pytest.raises(sop.SopError):
        sop.surrogate_file_read(tmp_path / "missing.ckpt", n)
