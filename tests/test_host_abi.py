"""Host-side logic behind the C ABI, exercised on CPU through the binding without any CUDA
call: argument validation that returns before the device is touched, the serving form's
request footprint model, the launch-shape table of the apply tuner, and the binding's
argument marshalling."""
import numpy as np
import pytest

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def req(dim=2, P=4, K=8, **kw):
    r = dict(dim=dim, P=P, nelem=(K,) * dim, lo=(0,) * dim, hi=(TWO_PI,) * dim, periodic=(1,) * dim,
             flow=imex.FLOW_TG2D if dim == 2 else imex.FLOW_TG3D, nu_kind=imex.NU_CONST, nu_params=[0.01])
    r.update(kw)
    return r


@pytest.mark.parametrize("bad", [dict(dim=4), dict(dim=1), dict(P=1), dict(P=9), dict(nelem=(0, 4)),
                                 dict(nelem=(4, -2))])
def test_footprint_rejects_invalid_requests(bad):
    r = req()
    r.update(bad)
    with pytest.raises(imex.ImexError) as e:
        imex.Server.footprint(**r)
    assert e.value.status == imex.EINVAL


def test_footprint_scales_with_the_nodes():
    """The admission model is linear in the velocity and pressure node counts: doubling the
    elements doubles it up to a fixed header; it grows with the degree and with d; and it
    holds at least the FP64 state, its stage sums and the solver vectors."""
    for dim, P in ((2, 3), (2, 8), (3, 5)):
        K = 6
        f1 = imex.Server.footprint(**req(dim, P, K))
        f2 = imex.Server.footprint(**req(dim, P, K, nelem=(2 * K,) + (K,) * (dim - 1)))
        c = 2 * f1 - f2                                 # the fixed part
        assert 0 <= c < 1e4
        assert abs((f2 - c) - 2 * (f1 - c)) <= 1e-9 * f2
        nv = K ** dim * (P + 1) ** dim
        # at least ten FP64 velocity-sized vectors per component, at most a few hundred
        assert 10 * 8 * dim * nv < f1 < 400 * 8 * dim * nv
    assert imex.Server.footprint(**req(2, 5)) > imex.Server.footprint(**req(2, 4))
    assert imex.Server.footprint(**req(3, 4, 8)) > imex.Server.footprint(**req(2, 4, 8))
    # the same mesh with data on Dirichlet sides and variable viscosity has the same footprint
    # model (the boundary data live in the per-instance table)
    a = imex.Server.footprint(**req(2, 6, 8))
    b = imex.Server.footprint(**req(2, 6, 8, periodic=(0, 0), flow=imex.FLOW_TGTRAVEL, nu_kind=imex.NU_VARXYT,
                                    bc_kind=imex.FLOW_TGTRAVEL, bc_params=[0.01],
                                    f_kind=imex.FORCE_TGTRAVEL_VARNU, f_params=[0.01]))
    assert a == b


@pytest.mark.parametrize("bad", [dict(dim=4), dict(P=1), dict(P=9), dict(nelem=(0, 3)), dict(hi=(0.0, TWO_PI)),
                                 dict(precision=7), dict(poisson=5)])
def test_create_rejects_invalid_meshes_before_the_device(bad):
    a = dict(dim=2, P=4, nelem=(3, 3), lo=(0, 0), hi=(TWO_PI, TWO_PI), periodic=(1, 1))
    a.update(bad)
    with pytest.raises(imex.ImexError) as e:
        imex.Context(**a)
    assert e.value.status == imex.EINVAL


def test_apply_variant_rules_and_table():
    """The launch shapes the tuner may fix: 0-3 for the FP32 3D applies of N = 7 and 9 (the
    fourth, one element more per block, exists only there), 0-2 elsewhere except the
    FP64 2D apply, which has two; the table reads back what was set."""
    ne = 123457                                          # an element count no context uses
    bad = [(3, 8, 1, 3), (3, 7, 0, 3), (2, 7, 1, 3), (2, 5, 0, 2), (3, 7, 1, 4), (3, 7, 1, -1), (4, 7, 1, 0),
           (3, 1, 1, 0), (3, 11, 1, 0)]
    for d, N, f32, v in bad:
        with pytest.raises(imex.ImexError):
            imex.set_apply_variant(d, N, f32, ne, v)
    with pytest.raises(imex.ImexError):
        imex.set_apply_variant(3, 7, 1, 0, 1)
    for d, N, f32, v in [(3, 7, 1, 3), (3, 9, 1, 3), (3, 8, 1, 2), (2, 5, 1, 2), (2, 5, 0, 1), (3, 4, 0, 0)]:
        imex.set_apply_variant(d, N, f32, ne, v)
    imex.set_apply_variant(3, 7, 1, ne, 1)               # a second call overwrites the entry
    got = {(t["d"], t["N"], t["fp32"]): t["variant"] for t in imex.tuning_info() if t["elements"] == ne}
    assert got == {(3, 7, True): 1, (3, 9, True): 3, (3, 8, True): 2, (2, 5, True): 2, (2, 5, False): 1,
                   (3, 4, False): 0}


def test_launch_counter_without_launches():
    """The library's launch counter is a host counter: none of the calls above launched."""
    n = imex.launch_count()
    assert n >= 0
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert n == 0


def test_binding_marshalling():
    """Host arrays reach the library as contiguous float64 (other dtypes and strides are
    copied), output arrays must already be writable contiguous float64, short buffers are
    refused before any call; parameter lists become float64 arrays; a request structure
    carries the mesh with the unused third direction set to one periodic element."""
    import ctypes
    p, dev, keep = imex._arr(np.arange(6, dtype=np.float32))
    assert dev == 0 and keep.dtype == np.float64 and np.array_equal(keep, np.arange(6.0))
    strided = np.arange(12.0)[::2]
    p, dev, keep = imex._arr(strided)
    assert keep.flags.c_contiguous and np.array_equal(keep, strided)
    assert ctypes.cast(p, ctypes.POINTER(ctypes.c_double))[3] == 6.0
    a = np.zeros(4)
    assert imex._arr(a, 4, writable=True)[2] is a              # no copy of a valid output
    for bad in (np.zeros(4, dtype=np.float32), np.zeros(8)[::2]):
        with pytest.raises(ValueError):
            imex._arr(bad, 4, writable=True)
    ro = np.zeros(4)
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        imex._arr(ro, 4, writable=True)
    with pytest.raises(ValueError):
        imex._arr(np.zeros(3), 4)
    assert imex._arr(None) == (None, 0, None)
    p, n, keep = imex._params([1, 2.5])
    assert n == 2 and keep.dtype == np.float64 and list(keep) == [1.0, 2.5]
    assert imex._params(()) == (None, 0, None)
    r = imex.Server.request(dim=2, P=5, nelem=(7, 3), lo=(0, -1), hi=(1, 2), periodic=(1, 0), flow=imex.FLOW_TG2D,
                            nu_params=[0.01], dt=0.002, nsteps=9)
    assert (r.dim, r.P, list(r.nelem), list(r.periodic)) == (2, 5, [7, 3, 1], [1, 0, 1])
    assert list(r.lo)[:2] == [0.0, -1.0] and list(r.hi)[:2] == [1.0, 2.0]
    assert r.nu_params[0] == 0.01 and r.dt == 0.002 and r.nsteps == 9
