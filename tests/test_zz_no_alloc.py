"""eels_matvec_dev_noalloc: the FFT matrix-vector product for callers that
cannot allocate device memory (for example latency-critical loops that must
not meet the allocator's synchronisation, or hosts whose own memory pool owns
the whole device).  Its FFT scratch is a fixed 64 MiB array inside the library.

Checked through the C ABI against eels_matvec_dev (context-owned scratch),
with the tolerances the matvec parity tests use, on two calls in a row (the
second call finds the first call's data still in the shared array).  This
file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda
    return eelsdda


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matvec_matches_context_matvec_twice(dd):
    import torch
    from paper_2208_01348_gb300 import inputs as I

    stream = torch.cuda.current_stream().cuda_stream
    ctx = dd.eels_create(0, stream)
    try:
        w = I.config_spectrum()
        g = w.grid
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        idx = np.array([0, 80, 199])
        dd.eels_prepare_operator(ctx, w.energies_eV[idx], w.eps_p[idx], w.eps_h[idx])
        n = dd.eels_num_dipoles(ctx)
        torch.manual_seed(3)
        for prec, dtype, tol in ((dd.EELS_MIXED, torch.complex64, 2e-5), (dd.EELS_FP64, torch.complex128, 1e-12)):
            x = torch.randn(3, 3, n, dtype=dtype, device="cuda")
            y_ref = torch.empty_like(x)
            dd.eels_matvec_dev(ctx, prec, x.data_ptr(), y_ref.data_ptr(), 3, stream)
            torch.cuda.synchronize()
            ref = y_ref.cpu().numpy()
            for _ in range(2):
                y = torch.full_like(x, float("nan"))
                dd.eels_matvec_dev_noalloc(ctx, prec, x.data_ptr(), y.data_ptr(), 3, stream)
                torch.cuda.synchronize()
                got = y.cpu().numpy()
                for s in range(3):
                    assert _rel(got[s], ref[s]) <= tol
        # a request beyond the fixed array is refused before anything runs
        many = np.linspace(0, 199, 11).astype(int)
        dd.eels_prepare_operator(ctx, w.energies_eV[many], w.eps_p[many], w.eps_h[many])
        x = torch.zeros(11, 3, n, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(dd.EelsError) as e:
            dd.eels_matvec_dev_noalloc(ctx, dd.EELS_FP64, x.data_ptr(), y.data_ptr(), 11, stream)
        assert e.value.code == dd.EELS_E_UNSUPPORTED and "fewer systems" in str(e.value)
    finally:
        dd.eels_destroy(ctx)
