"""The allocation-free reduction entry point against the context-based one.

imex_reduce_noalloc serves callers that cannot allocate device memory when they call
the library (another framework's memory pool owns the device, or allocation would
synchronise a hot loop, or the host forbids it after start-up).  It must give the same
results as imex_reduce on two calls in a row, because every call shares one fixed
device array of partial sums.  This file sorts last so that a run stopping at its
first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def test_noalloc_reduce_matches_context_reduce_twice():
    ctx = imex.Context(3, 3, (3, 2, 3), [0, 0, 0], [1, 1, 1], (1, 1, 1))
    n = ctx.dim * ctx.nvel
    for call, seed in enumerate((31, 32)):
        rng = np.random.default_rng(seed)
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        y = torch.from_numpy(rng.standard_normal(n)).cuda()
        if call == 1:
            x[5] = float("nan")
        torch.cuda.synchronize()
        for op, tol in ((imex.REDUCE_DOT, 1e-13), (imex.REDUCE_SUM, 1e-12), (imex.REDUCE_MAXABS, 0.0)):
            a = ctx.reduce(op, x, y if op == imex.REDUCE_DOT else None)
            b = imex.reduce_noalloc(op, x, y if op == imex.REDUCE_DOT else None)
            if np.isnan(a):
                assert np.isnan(b), (call, op)
            else:
                assert b == pytest.approx(a, rel=tol, abs=1e-13), (call, op, a, b)


def test_noalloc_reduce_rejects_sizes_above_its_limit():
    x = torch.zeros(imex.NOALLOC_MAX_N + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(imex.ImexError) as e:
        imex.reduce_noalloc(imex.REDUCE_SUM, x)
    assert e.value.status == imex.EINVAL
    assert imex.reduce_noalloc(imex.REDUCE_SUM, x[:imex.NOALLOC_MAX_N]) == 0.0
