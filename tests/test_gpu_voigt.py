"""The Voigt function as the kernels evaluate it (mpsa_voigt, through the C ABI) against the
FP64 oracle H = Re w(v + ia), per tier, on a (v, a) grid that spans every tier boundary."""
import numpy as np
import pytest

from oracle.voigt import H

pytestmark = pytest.mark.gpu

# relative-error bounds per tier (FP32 evaluation; derived from the tier truncation errors
# plus a few FP32 roundings: far <= 1e-6 + rounding, mid and core ~ 3e-6)
FP32_RTOL = 5e-6
FP64_RTOL = 1e-11


def grid():
    a = np.geomspace(1e-5, 30.0, 61)
    v = np.r_[0.0, np.geomspace(1e-3, 1e7, 700)]
    # points hugging the tier boundaries |z|^2 = 36 and 1600 and the rational-form switch
    extra_v = []
    for aa in a:
        for z2 in (36.0, 1600.0, 1000.0 * np.sqrt(2 + 2 * aa * aa)):
            for f in (1 - 1e-6, 1 + 1e-6):
                if z2 * f > aa * aa:
                    extra_v.append((np.sqrt(z2 * f - aa * aa), aa))
    V, A = np.meshgrid(v, a, indexing="ij")
    V, A = V.ravel(), A.ravel()
    ev = np.array(extra_v)
    return np.r_[V, ev[:, 0]], np.r_[A, ev[:, 1]]


def device_H(ctx, v, a, prec):
    import torch
    tv = torch.from_numpy(v).cuda()
    ta = torch.from_numpy(a).cuda()
    out = torch.empty_like(tv)
    ctx.voigt(tv, ta, out, precision=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_fp32_tiers_against_oracle():
    from paper_2105_13611_gb300 import binding
    ctx = binding.Context(0)
    v, a = grid()
    vf, af = v.astype(np.float32).astype(np.float64), a.astype(np.float32).astype(np.float64)
    g = device_H(ctx, vf, af, binding.PREC_FP32_COMPENSATED)
    o = H(vf, af)
    rel = np.abs(g / o - 1)
    z2 = vf * vf + af * af
    for name, m in (("core", z2 < 36), ("mid", (z2 >= 36) & (z2 < 1600)), ("far", z2 >= 1600)):
        assert m.any()
        assert rel[m].max() <= FP32_RTOL, (name, rel[m].max(), vf[m][np.argmax(rel[m])], af[m][np.argmax(rel[m])])
    ctx.close()


def test_fp64_tiers_against_oracle():
    from paper_2105_13611_gb300 import binding
    ctx = binding.Context(0)
    v, a = grid()
    g = device_H(ctx, v, a, binding.PREC_FP64)
    o = H(v, a)
    rel = np.abs(g / o - 1)
    assert rel.max() <= FP64_RTOL, (rel.max(), v[np.argmax(rel)], a[np.argmax(rel)])
    ctx.close()
