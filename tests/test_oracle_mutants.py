"""Planted mistakes in the oracle, on the CPU.

Each entry below is a plausible slip in oracle/oracle.cpp (a dropped term, a
wrong sign, a wrong weight or index, a min for a max).  The test builds the
oracle from a copy of the source with that one change, runs the oracle's pins
(tests/test_oracle_*.py, closed forms, invariants, independent assemblies and
brute force) against the build, and requires every such build to fail at
least one pin: the pins constrain the oracle, they do not merely restate it.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
PINS = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
              if f.startswith("test_oracle_") and f.endswith(".py") and f != os.path.basename(__file__))

# (name, text in oracle.cpp (exactly once), replacement)
MUTANTS = [
    ("fine mass matrix: off-diagonal h/4 instead of h/6",
     "    M(i, i + 1) += h / 6.0;\n    M(i + 1, i) += h / 6.0;",
     "    M(i, i + 1) += h / 4.0;\n    M(i + 1, i) += h / 4.0;"),
    ("mass matrix: diagonal h/2 instead of h/3 on the left node",
     "    M(i, i) += h / 3.0;",
     "    M(i, i) += h / 2.0;"),
    ("interpolation weights of the two coarse neighbours swapped",
     "      L.I(i, J - 1) = (b - t) / (b - a);\n      L.I(i, J) = (t - a) / (b - a);",
     "      L.I(i, J - 1) = (t - a) / (b - a);\n      L.I(i, J) = (b - t) / (b - a);"),
    ("projection without the fine mass matrix (P = Mc^-1 I^T)",
     "        for (int t = 0; t < L.n; ++t) s += L.I(t, a) * L.Mf(t, b);",
     "        for (int t = 0; t < L.n; ++t) s += L.I(t, a) * (t == b ? 1.0 : 0.0);"),
    ("coefficient without the interpolant (d = u)",
     "        double d = u.at(i, j, k) - E.at(i, j, k);",
     "        double d = u.at(i, j, k);"),
    ("coarse correction subtracted in the decomposition",
     "  Grid z = project(D, L);\n  for (size_t t = 0; t < uc.v.size(); ++t) uc.v[t] += z.v[t];",
     "  Grid z = project(D, L);\n  for (size_t t = 0; t < uc.v.size(); ++t) uc.v[t] -= z.v[t];"),
    ("last node not kept on the coarse grid",
     "  if ((n - 1) % 2 != 0) c.push_back(n - 1);",
     "  if (false) c.push_back(n - 1);"),
    ("zero fill replaced by a fill of ones",
     "blk.at(i, j, k) = inside ? in.at(gi, gj, gk) : 0.0;",
     "blk.at(i, j, k) = inside ? in.at(gi, gj, gk) : 1.0;"),
    ("FP64 quantiser truncates instead of rounding half up",
     "    double y = std::fma(c, rq, 0.5);",
     "    double y = c * rq;"),
    ("error shares over N levels instead of N + 1",
     "  double t = (double)(N + 1);\n  double denom = t * A;",
     "  double t = (double)N;\n  double denom = t * A;"),
    ("global levels take the last tier instead of the strictest",
     "    tau_g = std::min(tau_g, taup[t]);",
     "    tau_g = taup[t];"),
    ("block tolerance ignores a looser ROI bound the wrong way (max)",
     "    if (roi) t = std::min(t, roi[b]);",
     "    if (roi) t = std::max(t, roi[b]);"),
    ("re-formed blocks keep the loosest tier",
     "                v = std::min(v, t[r][(size_t)((i0 * a.nb[1] + i1) * a.nb[2] + i2)]);",
     "                v = std::max<uint8_t>(v == 255 ? (uint8_t)0 : v, t[r][(size_t)((i0 * a.nb[1] + i1) * a.nb[2] + i2)]);"),
    ("Huffman merging takes an internal node before a leaf of equal weight",
     "    if (lp < n && (qp >= qe || w[lp] <= w[qp])) return lp++;",
     "    if (lp < n && (qp >= qe || w[lp] < w[qp])) return lp++;"),
    ("canonical codes ordered by descending length",
     "  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len[a] < len[b]; });",
     "  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len[a] > len[b]; });"),
    ("round-off margin dropped",
     "  b.margin = ((kKappa * eps) * (double)(N + 1)) * max_abs;",
     "  b.margin = 0.0;"),
]


def _run_mutant(tmp, k, old, new):
    src = open(SRC).read()
    if src.count(old) != 1:
        return "text not found exactly once"
    d = os.path.join(tmp, "m%02d" % k)
    os.makedirs(d, exist_ok=True)
    cpp = os.path.join(d, "oracle.cpp")
    with open(cpp, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(d, "liboracle.so")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", cpp,
                        "-o", so], capture_output=True, text=True)
    if r.returncode != 0:
        return "does not compile: " + r.stderr[-300:]
    env = dict(os.environ, OR_LIBRARY=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode == 0:
        return "survived"
    first = [l.split(" ", 1)[1].split(" - ")[0] for l in r.stdout.splitlines() if l.startswith(("FAILED ", "ERROR "))]
    return "killed by " + (first[0] if first else "a crash")


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        futs = [ex.submit(_run_mutant, str(tmp_path), k, old, new) for k, (_, old, new) in enumerate(MUTANTS)]
        res = [f.result() for f in futs]
    bad = [(name, r) for (name, _, _), r in zip(MUTANTS, res) if not r.startswith("killed")]
    assert not bad, bad


def test_pins_pass_on_the_unmodified_oracle_build(tmp_path):
    """The same harness on an unmodified copy passes (so a kill above is the
    planted change, not the harness)."""
    assert _run_mutant(str(tmp_path), 99, "namespace {", "namespace {") == "survived"


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
