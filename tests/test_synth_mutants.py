"""The generator checks catch plausible mistakes in the input generator.

Each case plants one slip in a copy of synth/__init__.py -- the focal
length, the principal point, the scale of w, the chord factor, the phantom
rotation, a half-pixel shift, the tilt size, the arc, the phantom extent --
and runs tests/test_synth.py against that copy in a separate process.  Every
mutant must fail at least one check; the unmutated copy must pass them all.
Only host code is mutated; nothing here touches a GPU.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "synth", "__init__.py")

MUTANTS = {
    "focal length from SID": ("f = cfg.sdd / cfg.pixel", "f = cfg.sid / cfg.pixel"),
    "u0 from the detector height": ("u0 = (cfg.det_w - 1) / 2.0", "u0 = (cfg.det_h - 1) / 2.0"),
    "w not scaled by SID": ("P /= np.linalg.norm(P[2, :3]) * cfg.sid", "P /= np.linalg.norm(P[2, :3])"),
    "half chord": ("line += dens[e] * 2.0 * torch.sqrt(disc) / A", "line += dens[e] * torch.sqrt(disc) / A"),
    "phantom rotation transposed": ("p = (S - cen[e]) @ Q / ax[e]", "p = (S - cen[e]) @ Q.T / ax[e]"),
    "rays through pixel corners": ("cu = ((mm.view(1, 1, W) - u0) / f)", "cu = ((mm.view(1, 1, W) + 0.5 - u0) / f)"),
    "tilts three times too large": ("R = R @ T.T", "R = R @ T.T @ T.T @ T.T"),
    "full circle instead of 200 degrees": ("np.linspace(0.0, cfg.arc_deg, n)", "np.linspace(0.0, 360.0, n)"),
    "ellipsoids reach past the field of view": ("rmax = 90.0 - axes[i].max()", "rmax = 90.0"),
}

_RUNNER = (
    "import sys; sys.path.insert(0, {pkg!r}); import synth; "
    "assert synth.__file__.startswith({pkg!r}), synth.__file__; "
    "import pytest; sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', {tests!r}]))"
)


def _run(tmp_path, name, text):
    pkg = tmp_path / name
    (pkg / "synth").mkdir(parents=True)
    (pkg / "synth" / "__init__.py").write_text(text)
    code = _RUNNER.format(pkg=str(pkg), tests=os.path.join(HERE, "test_synth.py"))
    return subprocess.run([sys.executable, "-c", code], cwd=str(pkg), capture_output=True, text=True,
                          timeout=600)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found once"
    r = _run(tmp_path, "mutant", src.replace(old, new))
    assert r.returncode == 1, f"{name}: not caught (rc {r.returncode})\n{r.stdout[-2000:]}{r.stderr[-2000:]}"


def test_unmutated_copy_passes(tmp_path):
    r = _run(tmp_path, "plain", open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
