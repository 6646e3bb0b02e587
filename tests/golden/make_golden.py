"""Write the oracle's expected values for the full-size parity tests.

Calls only the oracle (oracle/) and the seeded input generators (synth/); no
value here comes from the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py protein40k      # ~15 min on 8 cores
    python tests/golden/make_golden.py multisurface400  # ~30 min on 8 cores

protein40k.json: the 2,000-atom synthetic protein (40,144 panels, K = 3,
K_fine = 19, thres = 2): the solvation energy of Eq. solv from the dense
matrix-free operator solved by GMRES to a relative residual of 1e-8, and the
operator (Eq. matrix, both row blocks) applied to a seeded vector on sampled
rows, once exactly (dense rule) and once by the oracle's treecode (Sec. 2.3,
theta = 0.5, P = 6, ncrit = 300: direct moments, jet coefficients).

multisurface400.json: the reduced multi-surface molecule (400 atoms, two
cavities, Stern layer; Sec. 2.2 "Multi-surface problems"): the energy of each
of its four model variants (single, cavity, Stern, full), and the full
variant's operator on sampled rows of every surface.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cdense  # noqa: E402
from oracle import formulation as F  # noqa: E402
from oracle.treecode import TreecodeOracle  # noqa: E402
from synth import configs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-8
X_SEED = 12345
ROW_SEED = 54321


def mesh_fingerprint(problem):
    """Exact topology hash and vertex checksums of every surface."""
    out = []
    for s in problem["surfaces"]:
        v = np.asarray(s["verts"], dtype=np.float64)
        t = np.ascontiguousarray(np.asarray(s["tris"], dtype=np.int32))
        out.append(dict(n_panels=int(t.shape[0]), n_verts=int(v.shape[0]),
                        tris_sha256=hashlib.sha256(t.tobytes()).hexdigest(),
                        verts_sum=float(v.sum()), verts_sumsq=float((v * v).sum())))
    return out


def seeded_vector(problem):
    n = 2 * configs.panel_count(problem)
    return np.random.default_rng(X_SEED).normal(size=n)


def sampled_rows(problem, per_surface):
    rng = np.random.default_rng(ROW_SEED)
    return [np.sort(rng.choice(n, min(per_surface, n), replace=False)) for n in F.n_panels(problem)]


def _log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def _rows_json(out, rows):
    return [dict(rows=rows[s].tolist(), inner=out[(s, 0)].tolist(), outer=out[(s, 1)].tolist())
            for s in range(len(rows))]


def energy(problem):
    t = time.time()
    r = cdense.solve(problem, tol=TOL, precond=True)
    _log(f"dG = {r['dG']:.12f} kJ/mol, {r['iters']} iterations, residual {r['resid']:.2e}")
    return dict(dG=r["dG"], iterations=int(r["iters"]), residual=float(r["resid"]),
                seconds=time.time() - t)


def protein40k():
    d = configs.protein_problem()
    x = seeded_vector(d)
    rows = sampled_rows(d, 200)
    _log("dense operator on sampled rows")
    dense = cdense.DenseOperator(d).apply(x, {0: rows[0]})
    _log("oracle treecode on sampled rows")
    tc = TreecodeOracle(d, dict(theta=0.5, P=6, ncrit=300))
    tree = tc.matvec(x, {0: rows[0]})
    _log("solve")
    out = dict(workload="synthetic protein, 2,000 atoms (seed 2), 40,144 panels",
               params=dict(K=3, K_fine=19, N_k=5, thres=2.0), gmres_tol=TOL,
               mesh=mesh_fingerprint(d), x_seed=X_SEED,
               dense_rows=_rows_json(dense, rows),
               treecode=dict(theta=0.5, P=6, ncrit=300, rows=_rows_json(tree, rows)),
               **energy(d))
    return out


def multisurface400():
    variants = configs.reduced_model_variants()
    out = dict(workload="reduced multi-surface molecule: " + json.dumps(configs.REDUCED_MULTISURFACE),
               params=dict(K=3, K_fine=19, N_k=5, thres=2.0), gmres_tol=TOL, x_seed=X_SEED, variants={})
    full = variants["full"]
    x = seeded_vector(full)
    rows = sampled_rows(full, 60)
    _log("full variant: dense operator on sampled rows")
    dense = cdense.DenseOperator(full).apply(x, {s: r for s, r in enumerate(rows)})
    out["full_dense_rows"] = _rows_json(dense, rows)
    for name, d in variants.items():
        _log(f"variant {name}: {configs.panel_count(d)} panels")
        out["variants"][name] = dict(mesh=mesh_fingerprint(d), **energy(d))
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["protein40k", "multisurface400"]
    for w in which:
        t0 = time.time()
        res = dict(globals()[w](), generated_by="tests/golden/make_golden.py " + w,
                   host_cores=len(os.sched_getaffinity(0)), total_seconds=None)
        res["total_seconds"] = time.time() - t0
        with open(os.path.join(HERE, w + ".json"), "w") as f:
            json.dump(res, f, indent=1)
        _log(f"wrote {w}.json in {res['total_seconds']:.0f} s")
