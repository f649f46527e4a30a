"""The full deviance of mixed-precision handles, whose eta comes from the block
step's split-BF16 tensor-core products (deviance_tc), against the FP64 oracle
at identical parameters (Table S1; App. B for the negative binomial).

Bar, from the arithmetic: each BF16 pair hi + lo carries a factor to within
2^-18 of its value, so the three products give eta to within ~1.2e-5 of
sum_k |L_ik R_jk|; an entry's deviance moves by |dD/deta| times that, with
signs that do not line up, and the FP32 unit deviances add ~1e-7 of the
total (as for the CUDA-core kernel). The totals are held to 2e-6 relative
(the CUDA-core kernel's own bar is 1e-6), and the tensor-core kernel to the
CUDA-core kernel (GMF_FLAG_SIMT_DEVIANCE) on the same parameters likewise.
Cases: ragged tiles in both directions, 16- and 32-bit counts, K up to 55
(two 128-byte operand atoms), weights, per-gene shapes, Poisson, counts far
above the log tables (the ratio form), and matrices with several tiles per
CTA of the persistent launch."""
import numpy as np
import pytest

from tests.test_gpu_parity import Pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


CASES = {
    # name: (n, m, p, q, d, family, nb_row, nb_col, extra)
    "nb_uint16_ragged_d20": (1100, 904, 3, 1, 20, "negbin", 512, 256, dict(y_dtype="uint16", zero_frac=0.9)),
    "nb_int32_ragged": (700, 452, 3, 1, 7, "negbin", 128, 96, dict(zero_frac=0.85)),
    "nb_weights_moments": (700, 456, 3, 1, 7, "negbin", 128, 96, dict(zero_frac=0.85, weights=True, alpha_mode=1)),
    "poisson_uint16": (600, 264, 2, 1, 5, "poisson", 128, 128, dict(y_dtype="uint16")),
    "nb_d50_two_atoms": (520, 384, 3, 1, 50, "negbin", 256, 128, dict(y_dtype="uint16", zero_frac=0.8)),
    "nb_large_counts": (400, 392, 3, 1, 6, "negbin", 128, 128, dict(y_dtype="uint16", zero_frac=0.2)),
    "poisson_large_counts": (400, 392, 2, 1, 6, "poisson", 128, 128, dict(zero_frac=0.02)),
    "nb_many_tiles_per_cta": (6000, 3000, 3, 1, 20, "negbin", 2048, 1024, dict(y_dtype="uint16", zero_frac=0.9)),
}


def _simt_twin(gmf, P, nb_row, nb_col):
    """The same handle type and parameters, deviance by the CUDA-core kernel."""
    mdl = gmf.Model(torch.from_numpy(P.prob.Y).cuda(), P.prob.X, P.prob.Z, P.prob.offset, P.start,
                    family=P.prob.family, nb_row=nb_row, nb_col=nb_col, row_perm=P.rp, col_perm=P.cp,
                    settings=P.settings, precision="mixed", flags=gmf.GMF_FLAG_SIMT_DEVIANCE,
                    W=None if P.W is None else torch.from_numpy(P.W).cuda())
    mdl.set_params(P.ref_params())
    return mdl


@pytest.mark.parametrize("case", list(CASES))
def test_tensor_core_deviance_at_identical_parameters(gmf, oracle_mod, case):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES[case]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, seed=11, precision="mixed", **extra)
    if "large_counts" in case:
        assert int(P.prob.Y.max()) >= 256 and (P.prob.Y >= 32).mean() > 0.1   # the ratio form carries much of it
    # parameters after one epoch of the oracle: not the generating law, so residuals of both signs
    P.ref.epoch(P.sigmas[0])
    P.gpu.set_params(P.ref_params())
    ref = P.ref.deviance()
    got = P.gpu.deviance()
    assert got == pytest.approx(ref, rel=2e-6), (got, ref, got / ref - 1)
    assert P.gpu.deviance() == got   # fixed assignment of tiles to CTAs: the same bits every call
    twin = _simt_twin(gmf, P, nbr, nbc)
    assert twin.deviance() == pytest.approx(got, rel=2e-6)


def test_tensor_core_deviance_async_and_per_gene_shapes(gmf, oracle_mod):
    """The device-side total (gmf_deviance_async) equals the synchronous one,
    and per-gene shapes (alpha_mode 2) take the variant that reads them."""
    P = Pair(gmf, oracle_mod, 1100, 704, 3, 1, 6, "negbin", 500, 384, seed=5, zero_frac=0.8, precision="mixed",
             alpha_mode=2)
    ac = P.prob.nb_size + 0.05
    P.ref.alpha_col = np.ascontiguousarray(ac, dtype=np.float64)
    P.ref._data.alpha_col = P.ref.alpha_col.ctypes.data
    P.gpu.set_gene_shapes(ac)
    P.gpu.set_params(P.ref_params())
    got = P.gpu.deviance()
    assert got == pytest.approx(P.ref.deviance(), rel=2e-6)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.gpu.deviance_async(out)
    torch.cuda.synchronize()
    assert float(out.item()) == got
