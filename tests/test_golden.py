"""Golden fixtures (tests/golden/): the settings the paper states in its
implementation details (Sec. 5.1) against the values the code uses, and a
regression record of the FP64 oracle on a few tiny inputs (written by
tests/golden/make_oracle_golden.py, which calls only the oracle)."""
import importlib.util
import inspect
import json
import os

import numpy as np

from paper_2510_07729_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_settings():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_settings.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("="))
            out[k] = float(v)
    return out


def test_optimisation_settings_match_the_paper():
    from oracle import optimize
    from paper_2510_07729_gb300 import sop
    p = paper_settings()
    assert optimize.LR_MAT == p["lr_environment_materials"]
    assert optimize.LR_SOP == p["lr_sop_textures"]
    assert optimize.LAM_LAM == p["lambda_lam"] and optimize.LAM_SOPS == p["lambda_sops"]
    sig = inspect.signature(sop.TextureOptimizer.__init__).parameters
    assert sig["lr_mat"].default == p["lr_environment_materials"]
    assert sig["lr_sop"].default == p["lr_sop_textures"]
    assert sig["lam_lam"].default == p["lambda_lam"] and sig["lam_sops"].default == p["lambda_sops"]


def test_object_workload_uses_the_paper_sop_settings():
    """The object workload's probe maps and light directions, and its probes'
    offset along the normals of the surface samples they were placed on."""
    p = paper_settings()
    c = I.make_object()
    assert c["R"] == p["sop_texture_resolution"] and c["S"] == p["sop_sampling_rays"]
    _, _, _, ppos, pnrm, samp, diag = I._object(1)
    # each probe sits at offset * size along its sample's normal
    back = ppos - p["sop_offset_fraction"] * diag * pnrm
    d = np.min(np.linalg.norm(back[:200, None, :] - samp[None, :, :], axis=2), axis=1)
    assert np.max(d) < 1e-9


def test_oracle_regression_record():
    """The oracle still computes what it computed when the record was
    written (a guard against unintended changes, not a pin)."""
    spec = importlib.util.spec_from_file_location("make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    now = mod.compute()
    rec = json.load(open(os.path.join(GOLDEN, "oracle_tiny.json")))
    for part in ("bake", "query"):
        for k, v in rec[part].items():
            a, b = np.asarray(now[part][k]), np.asarray(v)
            if a.dtype.kind in "iu":
                assert np.array_equal(a, b), (part, k)
            else:
                np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15, err_msg=f"{part} {k}")
    assert now["fps"] == rec["fps"]
