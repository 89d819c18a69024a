"""Reduced-precision storage of the atlas depth plane (the FP8 E4M3 depth of
the reduced-precision form; FP16 and BF16 beside it), through the C ABI:
the stored codes are the correctly rounded values of D / depth_scale, bit
for bit, with the quotient taken in float32 on both sides (the library
multiplies by the float32 reciprocal of depth_scale)."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def quotient(d, scale):
    inv = np.float32(1.0) / np.float32(scale)
    return (np.asarray(d, np.float32) * inv).astype(np.float32)


def round_bf16_bits(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def stored_interior(at, R):
    d = at.depth[:, 1:R + 1, 1:R + 1].contiguous()
    return d.view(torch.uint8 if d.element_size() == 1 else torch.int16).cpu().numpy()


@pytest.mark.parametrize("scale", [1.0, 1.37, 0.05])
def test_fp8_depth_pack_bit_exact(sop, orc, scale):
    rng = np.random.default_rng(3)
    P, R = 9, 8
    maps = I.synthetic_maps(rng, P, R)
    dep = rng.uniform(0, 3.0, (P, R, R)).astype(np.float32) * np.float32(scale)
    # values on the FP8 grid, halfway points (ties) and values past 448
    q = np.float32(scale)
    dep[0, 0, :4] = np.array([1.0625, 1.1875, 0.0, 500.0], np.float32) * q
    dep[1, 0, :3] = np.array([2.0 ** -9, 1.5 * 2.0 ** -9, 2.0 ** -10], np.float32) * q
    at = sop.make_atlas(cuda(rng.standard_normal((P, 3)).astype(np.float32)), R, depth_dtype=sop.SOP_FP8E4M3,
                        depth_scale=scale)
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(dep), at)
    torch.cuda.synchronize()
    got = stored_interior(at, R)
    want = orc.fp8_e4m3_bits(quotient(dep, scale))
    assert np.array_equal(got, want)
    # the border copies the interior by the border rule
    full = at.depth.view(torch.uint8).cpu().numpy()
    for jj in (0, R + 1):
        for ii in range(R + 2):
            si, sj = orc.oct_wrap(R, ii - 1, jj - 1)
            assert np.array_equal(full[:, jj, ii], want[:, sj, si])


@pytest.mark.parametrize("dtype", ["fp16", "bf16"])
def test_16bit_depth_pack_bit_exact(sop, dtype):
    rng = np.random.default_rng(4)
    P, R, scale = 5, 8, 1.9
    maps = I.synthetic_maps(rng, P, R)
    dep = rng.uniform(0, 4.0, (P, R, R)).astype(np.float32)
    dt = sop.SOP_F16 if dtype == "fp16" else sop.SOP_BF16
    at = sop.make_atlas(cuda(rng.standard_normal((P, 3)).astype(np.float32)), R, depth_dtype=dt, depth_scale=scale)
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(dep), at)
    torch.cuda.synchronize()
    got = stored_interior(at, R).view(np.uint16)
    qv = quotient(dep, scale)
    want = qv.astype(np.float16).view(np.uint16) if dtype == "fp16" else round_bf16_bits(qv)
    assert np.array_equal(got, want)


def test_fp8_bake_depth_is_the_rounded_fp32_depth(sop, orc):
    """The bake writes the FP8 depth plane from the same float32 D / scale
    as its float32 plane: the codes are that value correctly rounded, and
    the float32 plane meets the FP64 oracle's depth."""
    c = I.make_tiny()
    g = {k: cuda(v) for k, v in c["gauss"].items()}
    scale = 2.0
    a32 = sop.make_atlas(cuda(c["probe_pos"]), c["R"], depth_scale=scale)
    a8 = sop.make_atlas(cuda(c["probe_pos"]), c["R"], depth_dtype=sop.SOP_FP8E4M3, depth_scale=scale)
    sop.bake(g, a32, t_stop=0.0)
    sop.bake(g, a8, t_stop=0.0)
    torch.cuda.synchronize()
    R = c["R"]
    d32 = a32.depth[:, 1:R + 1, 1:R + 1].cpu().numpy()
    assert np.array_equal(stored_interior(a8, R), orc.fp8_e4m3_bits(d32))
    _, o_occ, o_dep, fl = orc.bake(c["gauss"], c["probe_pos"], R, t_stop=0.0)
    ok = (fl & (orc.FLAG_ORDER | orc.FLAG_ALPHA_MIN | orc.FLAG_TNEAR)) == 0
    # stored D / scale in float32 against the oracle's D / scale
    err = np.abs(d32[ok].astype(np.float64) - o_dep[ok] / scale)
    assert err.max() <= 1e-5 * max(np.abs(o_dep[ok] / scale).max(), 1e-3) + 4 * 2.0 ** -24 * 2.0
