"""The renderer's FP32 Gaussian tail against CUDA's FP64 erfc (torch.special.erfc on the GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tail(u):
    from paper_2008_05858_gb300 import binding as B

    out = torch.empty(u.shape, dtype=torch.float32, device="cuda")
    B.e2e_eval_tail(u.data_ptr(), u.numel(), out.data_ptr())
    torch.cuda.synchronize()
    return out


def test_tail_relative_error_is_a_few_ulp():
    g = torch.Generator(device="cuda").manual_seed(5)
    u = torch.cat([torch.linspace(-6.5, 6.5, 2_000_001, dtype=torch.float64, device="cuda"),
                   (torch.rand(4_000_000, dtype=torch.float64, device="cuda", generator=g) - 0.5) * 9.0])
    got = tail(u).double()
    ref = torch.special.erfc(u.abs())
    rel = ((got - ref).abs() / ref).max().item()
    assert rel < 6e-7, rel  # 10 FP32 ulp worst case (measured 5.2e-7)
    rms = (((got - ref) / ref) ** 2).mean().sqrt().item()
    assert rms < 1.2e-7, rms


def test_far_tail_relative_error_is_a_few_ulp():
    # the cheaper rational of the tail edges (one or more pixels from a stamp's centre), on the
    # range the planner admits it for (arguments >= 0.4 in log2 units, |u| >= 0.333)
    from paper_2008_05858_gb300 import binding as B

    g = torch.Generator(device="cuda").manual_seed(6)
    lo = 0.4 / 1.2011224087864498
    u = torch.cat([torch.linspace(lo, 6.5, 2_000_001, dtype=torch.float64, device="cuda"),
                   lo + torch.rand(4_000_000, dtype=torch.float64, device="cuda", generator=g) * (6.5 - lo)])
    u = torch.cat([u, -u])
    out = torch.empty(u.shape, dtype=torch.float32, device="cuda")
    B.e2e_eval_tail_far(u.data_ptr(), u.numel(), out.data_ptr())
    torch.cuda.synchronize()
    ref = torch.special.erfc(u.abs())
    rel = ((out.double() - ref).abs() / ref).max().item()
    assert rel < 6e-7, rel
    rms = (((out.double() - ref) / ref) ** 2).mean().sqrt().item()
    assert rms < 1.2e-7, rms


def test_tail_is_finite_and_monotone_far_out():
    u = torch.linspace(0.0, 60.0, 100_001, dtype=torch.float64, device="cuda")
    got = tail(u)
    assert torch.isfinite(got).all().item()
    assert (got[1:] <= got[:-1]).all().item()
    assert got[-1].item() == 0.0


def test_tail_uses_the_low_word_of_the_argument():
    # erfc(4 + d) for d below FP32 resolution at 4 (ulp 4.8e-7): ignoring the low word would
    # cost d * dln(erfc)/du ~ 8.3 d ~ 1.7e-6 relative at d = 2e-7
    d = torch.tensor([0.0, 1e-7, 2e-7, -1e-7, 2.3e-7], dtype=torch.float64, device="cuda")
    u = 4.0 + d
    assert (u.float().double() == 4.0).all().item()
    got = tail(u).double()
    ref = torch.special.erfc(u)
    assert ((got - ref).abs() / ref).max().item() < 5e-7
