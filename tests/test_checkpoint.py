"""Training checkpoints of the learned predictor (paper_1504_01441_b300/learned.py): the
flat file round-trips every field, and a truncated, corrupted or foreign file is refused.
The resume itself (bit-identical parameters) is a GPU test in test_gpu_learned.py."""
import numpy as np
import pytest


def _arrays(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=n).astype(np.float32) for _ in range(3)]


def test_round_trip(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_1504_01441_b300 import learned
    g = torch.Generator(device="cpu").manual_seed(5)
    torch.randint(0, 10, (7,), generator=g)
    theta, m, v = _arrays()
    path = str(tmp_path / "ck.bin")
    learned.write_checkpoint(path, theta, m, v, 42, 17, g.get_state().numpy().tobytes())
    ck = learned.read_checkpoint(path)
    for a, b in zip((theta, m, v), (ck["theta"], ck["m"], ck["v"])):
        assert a.tobytes() == b.tobytes()
    assert ck["adam_t"] == 42 and ck["step"] == 17
    # the restored generator continues the same stream
    g2 = torch.Generator(device="cpu")
    g2.set_state(torch.frombuffer(bytearray(ck["rng_state"]), dtype=torch.uint8))
    assert torch.equal(torch.randint(0, 1000, (20,), generator=g),
                       torch.randint(0, 1000, (20,), generator=g2))


def test_damaged_files_are_refused(tmp_path):
    from paper_1504_01441_b300 import learned
    theta, m, v = _arrays(64)
    path = str(tmp_path / "ck.bin")
    learned.write_checkpoint(path, theta, m, v, 1, 1, b"state")
    good = open(path, "rb").read()
    cases = {"flipped": bytearray(good), "truncated": good[:-9], "foreign": b"NOTACKPT" + good[8:]}
    cases["flipped"][100] ^= 0x40
    for name, data in cases.items():
        bad = str(tmp_path / f"{name}.bin")
        open(bad, "wb").write(bytes(data))
        with pytest.raises(ValueError):
            learned.read_checkpoint(bad)
    with pytest.raises(ValueError):
        learned.write_checkpoint(path, theta, m[:10], v, 1, 1, b"")
