"""Field checkpoints (paper_0807_0264_gb300.checkpoint): round trip bit for
bit for every array type, a readable header, refusal of foreign or truncated
files (CPU); a plain FP64 fix cut by a save and a load equals the
uninterrupted fix bit for bit (GPU)."""
import numpy as np
import pytest

from paper_0807_0264_gb300 import checkpoint, synth

torch = pytest.importorskip("torch")


def test_round_trip_is_bit_exact(tmp_path):
    rng = np.random.default_rng(5)
    arrays = {"U": torch.from_numpy(rng.standard_normal((1, 4, 2, 9, 12, 2))),
              "U32": torch.from_numpy(rng.standard_normal((2, 4, 2, 9, 12, 2)).astype(np.float32)),
              "Z": torch.from_numpy(rng.integers(-1, 2, size=(1, 4, 2, 12)).astype(np.int8)),
              "canon": synth.make_field((2, 2, 2, 6), 0.3, 1)}
    p = tmp_path / "f.mcg"
    h = checkpoint.save(p, (2, 2, 2, 6), arrays, {"sweeps": 17, "R": 1.25})
    h2, back = checkpoint.load(p)
    assert h2 == h and h2["meta"] == {"sweeps": 17, "R": 1.25}
    for k, a in arrays.items():
        x = a.numpy() if hasattr(a, "numpy") else a
        assert back[k].dtype == x.dtype and back[k].shape == x.shape
        assert np.array_equal(back[k], x)
    # little-endian on disk whatever the host
    with open(p, "rb") as f:
        f.readline()
        raw = f.read(8)
    assert np.frombuffer(raw, "<f8")[0] == arrays["U"].numpy().ravel()[0]
    _, tens = checkpoint.load(p, device="cpu")
    assert torch.equal(tens["U"], arrays["U"])


def test_refuses_foreign_and_truncated_files(tmp_path):
    p = tmp_path / "x"
    p.write_bytes(b'{"format": "other", "version": 1}\n')
    with pytest.raises(ValueError):
        checkpoint.load(p)
    p.write_bytes(b"\x00\x01not json\n")
    with pytest.raises(ValueError):
        checkpoint.load(p)
    q = tmp_path / "t.mcg"
    checkpoint.save(q, (2, 2, 2, 2), {"a": np.arange(100, dtype=np.float64)})
    q.write_bytes(q.read_bytes()[:-8])
    with pytest.raises(ValueError):
        checkpoint.load(q)


@pytest.mark.gpu
def test_fix_resumed_from_a_checkpoint_equals_the_uninterrupted_fix(tmp_path):
    from paper_0807_0264_gb300 import mcg

    dims = (4, 4, 4, 6)
    U0 = mcg.mcg_pack_links(torch.from_numpy(synth.make_field(dims, 0.6, 2)).unsqueeze(0).cuda(), dims)
    G0 = mcg.identity_gauge(dims)
    for solve32 in (0, 1):
        p = dict(tol=-1e300, check_every=3, reunit_every=3, fp64_solve32=solve32)
        Ua, Ga = U0.clone(), G0.clone()
        mcg.mcg_fix(Ua, Ga, dims, mcg.Params(max_sweeps=12, **p))
        Ub, Gb = U0.clone(), G0.clone()
        r = mcg.mcg_fix(Ub, Gb, dims, mcg.Params(max_sweeps=6, **p))
        f = tmp_path / f"half{solve32}.mcg"
        checkpoint.save(f, dims, {"U": Ub, "G": Gb}, {"sweeps": r["sweeps"][0], "R": r["R"][0]})
        del Ub, Gb
        h, arr = checkpoint.load(f, device="cuda")
        assert h["meta"]["sweeps"] == 6
        Uc, Gc = arr["U"].contiguous(), arr["G"].contiguous()
        mcg.mcg_fix(Uc, Gc, dims, mcg.Params(max_sweeps=6, **p))
        assert torch.equal(Uc, Ua) and torch.equal(Gc, Ga)
