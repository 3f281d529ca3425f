"""The host-side reader and writer of the MD checkpoint format (no GPU)."""
import numpy as np
import pytest

from paper_2303_03529_gb300 import checkpoint


def _state(rng, nat=4, kmax=3):
    n2 = 2 * nat
    return dict(n_atoms=nat, n2=n2, kmax=kmax, precision=1, l_resolved=0, md_step=17,
                mu=-4.9, mu_prev=-4.95, R=rng.random((nat, 3)), V=rng.random((nat, 3)),
                nhist=rng.random((kmax + 1, n2)), F=rng.random((nat, 3)), Kf=rng.random(n2),
                K0=-np.eye(n2))


def test_fnv1a64_published_vectors():
    # FNV-1a 64 of the empty string is the offset basis; of "a" the published value
    assert checkpoint.fnv1a64(b"") == 0xCBF29CE484222325
    assert checkpoint.fnv1a64(b"a") == 0xAF63DC4C8601EC8C


def test_round_trip_and_rejections(tmp_path):
    ck = _state(np.random.default_rng(0))
    p = tmp_path / "s.ckpt"
    checkpoint.write(p, ck)
    back = checkpoint.read(p)
    for k, v in ck.items():
        if isinstance(v, np.ndarray):
            np.testing.assert_array_equal(back[k], v)
        else:
            assert back[k] == v
    raw = bytearray(p.read_bytes())
    raw[-3] ^= 0x01
    (tmp_path / "bad.ckpt").write_bytes(bytes(raw))
    with pytest.raises(ValueError, match="hash"):
        checkpoint.read(tmp_path / "bad.ckpt")
    checkpoint.read(tmp_path / "bad.ckpt", verify=False)  # shape checks alone pass
    (tmp_path / "magic.ckpt").write_bytes(b"XXXXXXXX" + bytes(raw[8:]))
    with pytest.raises(ValueError, match="magic"):
        checkpoint.read(tmp_path / "magic.ckpt")
    (tmp_path / "short.ckpt").write_bytes(bytes(raw[:-8]))
    with pytest.raises(ValueError, match="size"):
        checkpoint.read(tmp_path / "short.ckpt")
    with pytest.raises(ValueError, match="shape"):
        checkpoint.write(tmp_path / "x.ckpt", dict(ck, Kf=np.zeros(3)))
