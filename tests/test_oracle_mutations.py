"""Mutation check of the oracle's pins (CPU only).

The pins must catch a plausible mistake anywhere in the oracle. Each case
copies oracle/, the input generators and the tests into a temporary
directory, plants ONE mistake in the copy's tsdf_oracle.cpp, and runs the
copy's pin module in a subprocess; the case passes when that run fails. The
mistakes are the kind a restatement of the paper could make -- a dropped
term, a flipped sign, a transposed operand or index, a missing step -- in
the fusion (Section 2.2 with reading R5: the half voxel of the centre map,
the rotation of the point and of the ray, the occlusion test, the dedupe,
the sample step, the local index, the colour channels) and in the extraction
(readings E1-E4:
the tetrahedra and their orientation, the case tables, the inside test, the
vertex position, the unobserved-corner rule, the quad diagonal).

Only the copy of oracle/ is changed; nothing of the CUDA library is built
or loaded.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "tsdf_oracle.cpp")).read()

FUSION = {
    "centre without the half voxel": (
        "half_minus_t[i] = std::fmaf(0.5f, v, -t[i]);", "half_minus_t[i] = -t[i];"),
    "sdf sign flipped": ("const float sdf = d - cc[2];", "const float sdf = cc[2] - d;"),
    "point rotated by R transposed": (
        "Pw[i] = std::fmaf(R[i][2], pcz, std::fmaf(R[i][1], pcy, std::fmaf(R[i][0], pcx, t[i])));",
        "Pw[i] = std::fmaf(R[2][i], pcz, std::fmaf(R[1][i], pcy, std::fmaf(R[0][i], pcx, t[i])));"),
    "centre map A = v R instead of v R^T": ("A[j][i] = v * R[i][j];", "A[j][i] = v * R[j][i];"),
    "ray rotation drops a term": (
        "Dw[i] = std::fmaf(R[i][2], dz, std::fmaf(R[i][1], dy, R[i][0] * dx));",
        "Dw[i] = std::fmaf(R[i][2], dz, R[i][0] * dx);"),
    "local index x and y swapped": (
        "floor_mod8(g[0]) + kEdge * floor_mod8(g[1])", "floor_mod8(g[1]) + kEdge * floor_mod8(g[0])"),
    "occlusion test sign flipped": ("(d2 - cc[2]) >= -tau", "(cc[2] - d2) >= -tau"),
    "no per-point dedupe": ("if (seen) continue;", ""),
    "projection drops cx": ("std::fmaf(fx, cc[0] * iz, cx)", "fx * (cc[0] * iz)"),
    "sample step 1.5 v": ("static_cast<float>(k - M) * v;", "static_cast<float>(k - M) * v * 1.5f;"),
    "red and blue swapped": ("B.r_sum[l] += static_cast<double>(col[0]) / 255.0;",
                             "B.r_sum[l] += static_cast<double>(col[2]) / 255.0;"),
}

EXTRACTION = {
    "a tetrahedron in negative orientation": ("{0, 1, 7, 5}", "{0, 1, 5, 7}"),
    "odd permutation in the lone-corner table": ("{1, 0, 3, 2}", "{1, 0, 2, 3}"),
    "odd permutation in the pair table": ("{0x5, 0, 2, 3, 1}", "{0x5, 0, 2, 1, 3}"),
    "inside includes zero": ("if (val[T[k]] < 0.0) m |= 1 << k;",
                             "if (val[T[k]] <= 0.0) m |= 1 << k;"),
    "vertex measured from the upper corner": (
        "const double t = val[lo] / (val[lo] - val[hi]);",
        "const double t = val[hi] / (val[hi] - val[lo]);"),
    "vertex at 1 - t": ("p[k] = plo + t * (phi - plo);", "p[k] = phi + t * (plo - phi);"),
    "corners without the half voxel": (
        "(static_cast<double>(g[k] + o_lo[k]) + 0.5) * v",
        "(static_cast<double>(g[k] + o_lo[k])) * v"),
    "a tetrahedron dropped": ("for (int t = 0; t < 6; ++t) {\n      const int* T",
                              "for (int t = 0; t < 5; ++t) {\n      const int* T"),
    "unobserved corners used": (
        "if (!value(gx + dx, gy + dy, gz + dz, val[c])) return;  // E1",
        "if (!value(gx + dx, gy + dy, gz + dz, val[c])) val[c] = 1.0;"),
    "quad split along the other diagonal": (
        "const int e1[3][2] = {{a, c}, {b, d}, {b, c}};",
        "const int e1[3][2] = {{a, d}, {b, d}, {b, c}};"),
}


def run_mutated(tmp_path, original, mutated, module):
    assert SRC.count(original) == 1, original
    work = tmp_path / "copy"
    skip = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o")
    for d in ("oracle", "paper_2608_08287_gb300", "tests"):
        shutil.copytree(os.path.join(ROOT, d), work / d, ignore=skip)
    (work / "oracle" / "tsdf_oracle.cpp").write_text(SRC.replace(original, mutated, 1))
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           os.path.join("tests", module)],
                          cwd=work, capture_output=True, text=True, timeout=900)


def assert_caught(r):
    last = (r.stdout.strip().splitlines() or [""])[-1]
    # exit status 1 with a failed test: a pin caught the mistake (a build
    # error of the mutated copy would show as an error, not as a failure)
    assert r.returncode == 1 and " failed" in last and "error" not in last, last


@pytest.mark.slow
@pytest.mark.parametrize("name", list(FUSION))
def test_fusion_pins_catch_the_mistake(tmp_path, name):
    assert_caught(run_mutated(tmp_path, *FUSION[name], "test_oracle_pins.py"))


@pytest.mark.slow
@pytest.mark.parametrize("name", list(EXTRACTION))
def test_extraction_pins_catch_the_mistake(tmp_path, name):
    assert_caught(run_mutated(tmp_path, *EXTRACTION[name], "test_oracle_extract.py"))


def test_unchanged_copy_passes(tmp_path):
    """The same procedure without a mistake passes: the failures above come
    from the planted mistakes, not from the copying."""
    r = run_mutated(tmp_path, "const float sdf = d - cc[2];", "const float sdf = d - cc[2];",
                    "test_oracle_extract.py")
    assert r.returncode == 0, r.stdout[-2000:]
