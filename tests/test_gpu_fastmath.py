"""The library's table-driven FP64 exp, expm1 and log1p, and its reciprocal and reciprocal square
root (used by the device model in place of CUDA's), against CUDA's own functions and against the
host C library, in units in the last place, over the argument ranges the model uses and across
their branch boundaries."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
MAX_ULP = 4.0


@pytest.fixture(scope="module")
def eec():
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as m
    return m


def _args(lo, hi, extra, n=400_000, seed=0):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.uniform(lo, hi, n), np.asarray(extra, float)])
    return x[(x >= lo) & (x <= hi)]


def _ulp(got, ref):
    return np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), np.finfo(float).tiny))


CASES = {
    "exp": (0, np.exp, [(-707.0, 709.0), (-40.0, 0.0), (-1e-3, 1e-3)],
            [0.0, -0.0, 1e-300, -706.9, 708.9, np.log(2) / 128, -np.log(2) / 128]),
    "expm1": (1, np.expm1, [(-38.0, 40.0), (-2 ** -6, 2 ** -6), (-1.0, 1.0), (-200.0, -30.0)],
              [0.0, 2 ** -6, -2 ** -6, np.nextafter(2 ** -6, 0), -38.0, -37.999, 40.0, 1e-300,
               -1e-300]),
    "log1p": (2, np.log1p, [(0.0, 1.0), (0.0, 2 ** -6), (2 ** -8, 2 ** -6), (0.0, 2 ** -9)],
              [0.0, 1.0, 2 ** -7, np.nextafter(2 ** -7, 0), 1e-300, 5e-324, 0.5, 2 ** -8,
               np.nextafter(2 ** -8, 1), 1 / 256 + 1 / 512, 2 ** -9, np.nextafter(2 ** -9, 0),
               1 / 512 + 1 / 1024]),
    "rcp": (3, lambda v: 1.0 / v, [(1e-3, 1e6), (1.0, 2.0), (-1e3, -1e-3)],
            [1.0, 2.0, 0.5, 1 + 2 ** -52, 2 - 2 ** -52, 3.0, -1.0, 1e-3, 1e6]),
    "rsqrt": (4, lambda v: 1.0 / np.sqrt(v), [(1e-6, 1e6), (1.0, 4.0), (1e-3, 1e-2)],
              [1.0, 2.0, 4.0, 0.25, 1 + 2 ** -52, 4 - 2 ** -50, 1e-6, 1e6]),
}
# the host reference of rcp and rsqrt is itself rounded twice (1 / sqrt(v)): allow 1 ulp more
HOST_SLACK = {"rsqrt": 1.0}


@pytest.mark.parametrize("name", list(CASES))
def test_fastmath_within_a_few_ulp_of_cuda_and_libm(eec, name):
    import torch
    fn, host, ranges, extra = CASES[name]
    for k, (lo, hi) in enumerate(ranges):
        x = _args(lo, hi, extra, seed=k)
        xt = torch.as_tensor(x, device="cuda")
        ours, ref = eec.eec_math_check(fn, xt)
        ours, ref = ours.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(ours))
        assert _ulp(ours, ref).max() <= MAX_ULP, (name, lo, hi, float(x[_ulp(ours, ref).argmax()]))
        assert _ulp(ours, host(x)).max() <= MAX_ULP + HOST_SLACK.get(name, 0.0), (name, lo, hi)
        if name in ("rcp", "rsqrt"):
            assert _ulp(ours, ref).max() <= 1.0, (name, lo, hi)
