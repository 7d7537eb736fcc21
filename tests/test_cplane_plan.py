"""The library's per-node strategy (csrc/cplane_strategy.h) replays the oracle's
decisions (CPU, no GPU).

For every node of oracle solves by the complex-plane strategy (Sec. 3.3) the
harness receives the node's starting disk, the Philox uniforms of each
attempt and the oracle's step outcomes (split, a chop with its rank, a
failure).  It must draw the same lines on the same disks -- random angles,
perpendicular lines after a chop, recentering after one or two chops -- and
end the node the same way (split, or a cluster with the same region).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

from oracle import cplane
from oracle.philox import uniform_pairs
from paper_1011_3077_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1011_3077_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path_factory.mktemp("plan") / "cplane_plan"
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-I", CSRC,
                           os.path.join(HERE, "harness", "cplane_plan.cpp"), "-o", str(exe)])
    return str(exe)


def _nodes(info):
    out = {}
    for rec in info.lines:
        out.setdefault(rec[0], []).append(rec)
    return out


def _replay(harness, seed, recs, m, max_fail):
    node = recs[0][0]
    c0, R0 = recs[0][5], recs[0][6]
    rows = []
    for rec in recs:
        att, outcome, rank = rec[1], rec[4], rec[7]
        u1, u2 = uniform_pairs(1, seed, cplane.PURPOSE_LINE, node, att)
        kind = {"split": 0, "chop": 1, "fail": 2}[outcome]
        rows.append("%.17g %.17g %d %d" % (float(u1[0]), float(u2[0]), kind, rank))
    inp = "%.17g %.17g %.17g %d %d %d\n" % (R0, c0.real, c0.imag, m, max_fail, len(rows))
    inp += "\n".join(rows) + "\n"
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout
    return [line.split() for line in out.strip().splitlines()]


CASES = [
    ("near_axis", lambda: workloads.near_axis(25), dict(seed=3, leaf_size=4)),
    ("jordan", lambda: workloads.jordan_hard(32), dict(seed=1, leaf_size=4, enclose=True)),
    ("normal", lambda: workloads.normal_complex(48)[0], dict(seed=3, leaf_size=8)),
]


def _loose(n=24):
    rng = np.random.default_rng(81)
    lam = 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    N = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), 1)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return Q @ (np.diag(lam) + 0.3 * N) @ Q.conj().T


CASES.append(("loose", _loose, dict(seed=4, leaf_size=6, enclose=True)))


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_node_plan_replays_the_oracle(harness, name, make, kw):
    A = make()
    T, U, w, info = cplane.schur_complex_plane(A, **kw)
    checked = 0
    clusters = [reg for _, _, reg in info.clusters]
    # replay every node that drew lines; the node size only tells a chop of
    # rank m (all eigenvalues right of the line) from one of rank 0
    for node, recs in _nodes(info).items():
        chop_ranks = [r[7] for r in recs if r[4] == "chop"]
        m = max(chop_ranks) if any(rk > 0 for rk in chop_ranks) else 10 ** 6
        lines = _replay(harness, kw["seed"], recs, m, 8)
        assert len(lines) == len(recs) + 1
        for rec, got in zip(recs, lines):
            assert got[0] == "line"
            wr, wi, t, cr, ci, R = map(float, got[1:])
            assert abs(complex(wr, wi) - rec[2]) <= 1e-15
            assert abs(t - rec[3]) <= 1e-13 * (1 + abs(rec[3]))
            assert abs(complex(cr, ci) - rec[5]) <= 1e-13 * (1 + abs(rec[5]))
            assert abs(R - rec[6]) <= 1e-13 * rec[6]
        end = lines[-1]
        if recs[-1][4] == "split":
            assert end[:2] == ["end", "split"]
        else:
            assert end[:2] == ["end", "cluster"]
            c_end, R_end = complex(float(end[2]), float(end[3])), float(end[4])
            assert any(abs(R_end - reg.R) <= 1e-13 * reg.R and abs(c_end - reg.c) <= 1e-13 * (1 + abs(reg.c))
                       and int(end[5]) == len(reg.halfplanes) for reg in clusters)
        checked += 1
    assert checked >= 1


@pytest.fixture(scope="module")
def children_harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path_factory.mktemp("kids") / "cplane_children"
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-I", CSRC,
                           os.path.join(HERE, "harness", "cplane_children.cpp"), "-o", str(exe)])
    return str(exe)


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_child_regions_replay_the_oracle(children_harness, name, make, kw):
    """After every split of the oracle's solves, the library's child_regions
    gives the children the same disks (each side's enclosing circle, or the
    block's own disk when that is not larger)."""
    A = make()
    T, U, w, info = cplane.schur_complex_plane(A, **kw)
    for node, reg, (wl, t), own, kids in info.split_regions:
        rows = ["%.17g %.17g %.17g %d" % (reg.c.real, reg.c.imag, reg.R, len(reg.halfplanes))]
        rows += ["%.17g %.17g %.17g" % (hw.real, hw.imag, ht) for hw, ht in reg.halfplanes]
        rows.append("%.17g %.17g %.17g" % (wl.real, wl.imag, t))
        rows += ["%.17g %.17g %.17g" % (c.real, c.imag, R) for c, R in own]
        out = subprocess.run([children_harness], input="\n".join(rows) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        for line, kid in zip(out[:2], kids):
            _, cr, ci, R = line.split()
            assert abs(complex(float(cr), float(ci)) - kid.c) <= 1e-13 * (1 + abs(kid.c))
            assert abs(float(R) - kid.R) <= 1e-13 * kid.R
