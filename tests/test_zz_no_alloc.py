"""fe_pairing_noalloc: the duality pairing for callers that cannot let the library allocate
device memory (their memory is all in their own pool, or an allocation's possible device
synchronization is not acceptable on their path).  It must agree with fe_pairing, the entry point
whose partial sums live in library-allocated scratch, on consecutive calls that share the static
scratch array.  This file is collected last so that a failure here comes after every other test."""
import gc
import math

import numpy as np
import pytest

from paper_2607_02335_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-14  # relative to sum |a_e b_e|, as in the fe_pairing parity test


def _pair(fe, gm, prec, a, b, fn):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    fn(gm.handle, prec, a, b, out)
    torch.cuda.synchronize()
    return out.item()


def test_noalloc_pairing_matches_pairing_on_consecutive_calls():
    from paper_2607_02335_gb300 import fe

    cases = [((6, 5, 4), 3, 11), ((3, 2, 2), 2, 12)]  # larger first: stale slots must not leak
    for m, p, seed in cases:
        gm = fe.Mesh(m, p, geom_mode=fe.FE_GEOM_AFFINE)
        a = torch.from_numpy(S.dual_cellwise(m, p, seed=seed)).cuda()
        b = torch.from_numpy(S.dual_cellwise(m, p, seed=seed + 100)).cuda()
        scale = float((a * b).abs().sum().item())
        for prec, (x, y) in ((fe.FE_F64, (a, b)), (fe.FE_F32, (a.float(), b.float()))):
            ref = _pair(fe, gm, prec, x, y, fe.fe_pairing)
            got = _pair(fe, gm, prec, x, y, fe.fe_pairing_noalloc)
            assert abs(got - ref) <= TOL * scale, (m, p, prec)
        gm.close()


def test_noalloc_pairing_rejects_meshes_beyond_its_scratch():
    from paper_2607_02335_gb300 import fe

    gm = fe.Mesh((64, 64, 33), 7, geom_mode=fe.FE_GEOM_AFFINE)  # 69,206,016 cell-wise entries
    assert gm.cellwise_len > 8192 * 8192
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fe.FeError) as e:
        fe.fe_pairing_noalloc(gm.handle, fe.FE_F64, small, small, out)
    assert e.value.status == fe.FE_ERR_INVALID and "static scratch limit" in str(e.value)
    gm.close()


@pytest.mark.parametrize("scale", [1.0, 1e-18, 1e18])
def test_noalloc_pairing_against_host_fp64_sum_without_allocating(scale):
    """Both pairings against an exactly rounded host sum (math.fsum) of the FP64 products, with
    the inputs scaled far outside the float range; the device's free memory and the caching
    allocator's reservation are the same before and after the no-allocation calls."""
    from paper_2607_02335_gb300 import fe

    m, p = (5, 4, 3), 3
    gm = fe.Mesh(m, p, geom_mode=fe.FE_GEOM_AFFINE)
    an = S.dual_cellwise(m, p, seed=21) * scale
    bn = S.dual_cellwise(m, p, seed=22) * scale
    ref = math.fsum((an * bn).tolist())
    mag = math.fsum(np.abs(an * bn).tolist())
    a = torch.from_numpy(an).cuda()
    b = torch.from_numpy(bn).cuda()
    _pair(fe, gm, fe.FE_F64, a, b, fe.fe_pairing_noalloc)  # first call on the device: set-up
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # meshes of earlier tests that the garbage collector frees inside the window would hand
    # device memory back (free memory up): collect them first and keep the collector off
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        for _ in range(2):
            fe.fe_pairing_noalloc(gm.handle, fe.FE_F64, a, b, out)
            torch.cuda.synchronize()
            assert abs(out.item() - ref) <= 1e-14 * mag, scale
        free1, reserved1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    finally:
        gc.enable()
    assert free1 >= free0 and reserved1 == reserved0  # nothing allocated on the device
    got = _pair(fe, gm, fe.FE_F64, a, b, fe.fe_pairing)
    assert abs(got - ref) <= 1e-14 * mag, scale
    gm.close()
