"""The pins of the two numpy/torch references (other distances and profiles;
the smooth vMF kernel) must catch plausible mistakes in them.

Each case copies the reference module, plants one mistake by a literal text
substitution, and runs that reference's pin file in a fresh interpreter with
the broken copy loaded in place of the module. The pins must fail for every
mutant. Nothing here touches a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KSHIFT = {
    "flat_exclusive": ("return (t <= 1.0).astype", "return (t < 1.0).astype"),
    "epanechnikov_in_distance": ("return np.maximum(0.0, 1.0 - t)", "return np.maximum(0.0, 1.0 - np.sqrt(t))"),
    "gaussian_without_half": ("return np.exp(-t / 2.0)", "return np.exp(-t)"),
    "euclid_h_not_squared": ("return D2 / (h * h)", "return D2 / h"),
    "cosine_distance_not_squared": ("return ((1.0 - Xn @ Pn.T) / h) ** 2", "return (1.0 - Xn @ Pn.T) / h"),
    "cosine_pixels_not_normalised": ("Pw = P / np.linalg.norm(P, axis=1, keepdims=True) if distance == COSINE else P",
                                     "Pw = P"),
    "cosine_mean_not_renormalised": ("Xn[ok] = Y[ok] / np.linalg.norm(Y[ok], axis=1, keepdims=True)",
                                     "Xn[ok] = Y[ok] / s[ok, None]"),
    "empty_window_moves": ("ok = s > 0", "ok = s >= 0"),
    "count_includes_zero_weights": ("(W > 0).sum(axis=1)", "(W >= 0).sum(axis=1)"),
    "run_extra_step": ("    for _ in range(T):", "    for _ in range(T + 1):"),
    "run_margin_ignored": ("            margin = min(margin, float(", "            margin = max(margin, float("),
    "run_seeds_not_normalised": ("        X = X / np.linalg.norm(X, axis=1, keepdims=True)\n", ""),
}

VMF = {
    "not_renormalised": ("X = Y / torch.linalg.norm(Y, dim=1, keepdim=True)", "X = Y"),
    "weight_sign": ("W = torch.exp(kappa * (X @ P.T))", "W = torch.exp(-kappa * (X @ P.T))"),
    "kappa_halved": ("W = torch.exp(kappa * (X @ P.T))", "W = torch.exp(0.5 * kappa * (X @ P.T))"),
    "pixels_normalised": ("Y = W @ P", "Y = W @ (P / torch.linalg.norm(P, dim=1, keepdim=True))"),
    "extra_step": ("    for _ in range(T):", "    for _ in range(T + 1):"),
    "objective_sign": ("return torch.exp(kappa * (X @ P.T)).sum(dim=1)", "return torch.exp(-kappa * (X @ P.T)).sum(dim=1)"),
    "loss_mean": ("return ((vmf_forward(P, X0, kappa, T) - target) ** 2).sum()",
                  "return ((vmf_forward(P, X0, kappa, T) - target) ** 2).mean()"),
    "vjp_upstream_negated": ("grad_outputs=G)", "grad_outputs=-G)"),
    "vjp_outputs_swapped": ("return XT.detach(), gP.detach(), gX.detach()",
                            "return XT.detach(), gX.detach(), gP.detach()"),
}

# load the broken copy as oracle.<name>, then run the pin file against it
BOOT = """
import importlib.util, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle
spec = importlib.util.spec_from_file_location("oracle.{name}", {path!r})
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.{name}"] = mod
spec.loader.exec_module(mod)
setattr(oracle, "{name}", mod)
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", {pins!r}]))
"""


def _run_mutant(module, pins, old, new, tmp_path):
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    path = tmp_path / (module + ".py")
    path.write_text(src.replace(old, new))
    boot = BOOT.format(root=ROOT, tests=os.path.join(ROOT, "tests"), name=module, path=str(path),
                       pins=os.path.join(ROOT, "tests", pins))
    return subprocess.run([sys.executable, "-c", boot], cwd=ROOT, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(KSHIFT))
def test_kshift_pins_catch_mutant(name, tmp_path):
    r = _run_mutant("kshift_ref", "test_kshift_oracle_pins.py", *KSHIFT[name], tmp_path)
    assert r.returncode == 1, f"pins did not catch mutant {name} (rc {r.returncode}):\n{r.stdout[-2000:]}{r.stderr[-2000:]}"


@pytest.mark.parametrize("name", sorted(VMF))
def test_vmf_pins_catch_mutant(name, tmp_path):
    r = _run_mutant("vmf_ref", "test_vmf_oracle_pins.py", *VMF[name], tmp_path)
    assert r.returncode == 1, f"pins did not catch mutant {name} (rc {r.returncode}):\n{r.stdout[-2000:]}{r.stderr[-2000:]}"


def test_unmutated_copies_pass(tmp_path):
    """The harness itself: an unchanged copy passes both pin files."""
    for module, pins in (("kshift_ref", "test_kshift_oracle_pins.py"), ("vmf_ref", "test_vmf_oracle_pins.py")):
        r = _run_mutant(module, pins, "from __future__ import annotations", "from __future__ import annotations",
                        tmp_path)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
