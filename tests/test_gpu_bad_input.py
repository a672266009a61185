"""Input validation through the C ABI: a caller's field with one non-finite
entry, or one link off SU(3) (scaled by 1.01), is refused with MCG_BAD_INPUT
by every entry point of the method, before any GPU work on it (the field is
left as it was), and the message names the first failing matrix.  The
corruption is made on the host; nothing on the GPU faults."""
import numpy as np
import pytest

from paper_0807_0264_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = (4, 4, 4, 6)


@pytest.fixture(scope="module")
def mcg():
    from paper_0807_0264_gb300 import mcg as m

    return m


def site_index(dims, x, y, z, t):
    return x + dims[0] * (y + dims[1] * (z + dims[2] * t))


def corrupted(kind):
    U = synth.make_field(DIMS, 0.5, 3)
    x = site_index(DIMS, 1, 2, 3, 4)  # parity (1+2+3+4) % 2 = 0, in-parity index x // 2
    if kind == "nan":
        U[x, 2, 1, 0] = complex(np.nan, 0.0)
    elif kind == "inf":
        U[x, 2, 0, 0] = complex(0.0, np.inf)
    else:
        U[x, 2] *= 1.01
    return U, x // 2


def expect_bad(mcg, fn, *args, where="mu 2, parity 0", finite_only=False, **kw):
    with pytest.raises(mcg.MCGError) as e:
        fn(*args, **kw)
    assert e.value.code == 4, str(e.value)
    msg = str(e.value)
    what = "non-finite entries" if finite_only else "not finite or not in SU(3)"
    assert what in msg and where in msg, msg
    return msg


@pytest.mark.parametrize("kind", ["nan", "inf", "scaled"])
@pytest.mark.parametrize("prec", [0, 1])
def test_method_entry_points_refuse_bad_links(mcg, kind, prec):
    U, s = corrupted(kind)
    Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), DIMS, prec)
    before = Ud.clone()
    Gd = mcg.identity_gauge(DIMS, 1, prec)
    where = f"mu 2, parity 0, in-parity site {s})"
    expect_bad(mcg, mcg.mcg_fix, Ud, Gd, DIMS, mcg.Params(tol=1e-10, max_sweeps=10), where=where)
    assert torch.equal(Ud.nan_to_num(), before.nan_to_num())  # refused before any work on it
    expect_bad(mcg, mcg.mcg_smear, Ud, DIMS, 0.1, 1.0, 2, where=where)
    if kind == "scaled":  # a finite link off SU(3) still has a sector
        mcg.mcg_center_project(Ud, DIMS)
    else:
        expect_bad(mcg, mcg.mcg_center_project, Ud, DIMS, where=where, finite_only=True)
    expect_bad(mcg, mcg.mcg_precondition_fix, Ud, Gd, DIMS, mcg.Params(tol=1e-10, max_sweeps=10), where=where)
    if prec == 0:
        expect_bad(mcg, mcg.mcg_precondition_levels, Ud, DIMS, [0, 2], mcg.Params(tol=1e-10, max_sweeps=10),
                   where=where)
        expect_bad(mcg, mcg.mcg_anneal, Ud, Gd, DIMS, [1.0], where=where)
    expect_bad(mcg, mcg.mcg_fix_batch, [Ud], [Gd], [DIMS], mcg.Params(tol=1e-10, max_sweeps=10), where=where)


def test_bad_transform_is_refused(mcg):
    U = synth.make_field(DIMS, 0.5, 3)
    Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), DIMS)
    G = synth.random_gauge(DIMS, 1)
    x = site_index(DIMS, 0, 1, 0, 0)  # parity 1
    G[x, 2, 2] = complex(np.nan, np.nan)
    Gd = mcg.mcg_pack_gauge(torch.from_numpy(G).unsqueeze(0).cuda(), DIMS)
    expect_bad(mcg, mcg.mcg_fix, Ud, Gd, DIMS, mcg.Params(tol=1e-10, max_sweeps=10),
               where=f"parity 1, in-parity site {x // 2})")


def test_clean_fields_pass_and_small_drift_is_accepted(mcg):
    """SU(3) fields pass, including FP32 copies and links off unitarity by
    1e-9 (rounding-level drift of stored configurations)."""
    U = synth.make_field(DIMS, 0.5, 3)
    U[5, 1] *= 1 + 1e-9
    for prec in (0, 1):
        Ud = mcg.mcg_pack_links(torch.from_numpy(U).unsqueeze(0).cuda(), DIMS, prec)
        Gd = mcg.identity_gauge(DIMS, 1, prec)
        mcg.mcg_fix(Ud, Gd, DIMS, mcg.Params(tol=1e-10, max_sweeps=5))
        mcg.mcg_center_project(Ud, DIMS)
