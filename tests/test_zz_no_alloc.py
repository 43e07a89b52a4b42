"""The inversion entry point that allocates nothing, against the allocating path.

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator, or their steady-state loop must not block on the device), so the
library offers ctaux_invert_noalloc, whose scratch is a static device array.
This test feeds it the FP64 N^{-1} of two configurations in a row and checks
the inverse and log-determinant against what the context path (set_config,
which rebuilds N with the allocating FP64 recomputation) produces, within the
FP64 tolerance of the other parity tests.  It lives in a file of its own that
pytest collects last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from parity import oracle_for
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pk = pytest.importorskip("paper_1010_3690_gb300")


def _device_colmajor(a):
    # row-major storage of a^T is column-major storage of a
    return torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda")


def test_noalloc_inversion_matches_allocating_path_on_two_calls():
    from paper_1010_3690_gb300 import ctaux
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ch = configs.cube8(K=16.0, k_max=32, capacity=512)
    for seed, n in ((1, 300), (2, 137)):        # two calls in a row, the second smaller
        cfg = configs.synthetic_configuration(ch, n, seed=seed)
        oc = oracle_for(ch)
        oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
        with pk.Context([ch]) as ctx:
            ctx.set_config(0, cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
            ref = [ctx.get_N(0, spin) for spin in (0, 1)]
            ref_logdet = ctx.stats(0)["logdet"]
        for spin in (0, 1):
            a = _device_colmajor(oc.ninv(spin))
            out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
            st = torch.cuda.current_stream().cuda_stream
            r = ctaux.ctaux_invert_noalloc(a.data_ptr(), n, out.data_ptr(), n, n,
                                           logdet.data_ptr(), st)
            assert r == 0
            torch.cuda.synchronize()
            inv = out.cpu().numpy().T
            np.testing.assert_allclose(inv, ref[spin], rtol=1e-9,
                                       atol=1e-12 * np.abs(ref[spin]).max())
            assert float(logdet.item()) == pytest.approx(ref_logdet[spin], rel=1e-10, abs=1e-9)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1010_3690_gb300 import ctaux
    m = 512 + 1                      # one more than CTAUX_NOALLOC_MAX_M
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = ctaux.ctaux_invert_noalloc(a.data_ptr(), m, a.data_ptr(), m, m)
    assert r == 4   # CTAUX_ECAPACITY, returned before any launch


@pytest.mark.parametrize("case", ["lda_above_m", "m_at_the_limit", "tiny_scale_with_zero"])
def test_noalloc_leading_dimensions_limit_and_scale(case):
    """Padded leading dimensions, the largest supported order, and a matrix
    scaled far below float32 range whose first column starts with an exact
    zero (the pivot search orders float64 magnitudes), against numpy."""
    from paper_1010_3690_gb300 import ctaux
    ch = configs.cube8(K=16.0, k_max=32, capacity=600)
    n = {"lda_above_m": 200, "m_at_the_limit": 512, "tiny_scale_with_zero": 150}[case]
    cfg = configs.synthetic_configuration(ch, n, seed=11)
    oc = oracle_for(ch)
    oc.set_config(cfg["tau"], cfg["site"], cfg["s"], cfg["birth"], cfg["t"])
    A = oc.ninv(0)
    scale = 1.0
    if case == "tiny_scale_with_zero":
        A = A.copy()
        A[0, 0] = 0.0
        scale = 1e-300
    A = A * scale
    lda = n + 37 if case == "lda_above_m" else n
    ldi = n + 5 if case == "lda_above_m" else n
    host = np.zeros((n, lda))          # column j of A in host[j, :n]
    host[:, :n] = A.T
    a = torch.tensor(host, dtype=torch.float64, device="cuda")
    out = torch.full((n, ldi), float("nan"), dtype=torch.float64, device="cuda")
    logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = ctaux.ctaux_invert_noalloc(a.data_ptr(), lda, out.data_ptr(), ldi, n, logdet.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert r == 0
    torch.cuda.synchronize()
    inv = out.cpu().numpy()[:, :n].T
    ref = np.linalg.inv(A)
    assert np.all(np.isfinite(inv))
    np.testing.assert_allclose(inv, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    sign, ld_ref = np.linalg.slogdet(A)
    assert float(logdet.item()) == pytest.approx(ld_ref, rel=1e-10, abs=1e-8)
