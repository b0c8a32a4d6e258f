"""Oracle Newton solutions of the two slab workloads, stored for the GPU
parity tests.

The oracle's load-stepped Newton iteration (Section 2, Eq. (tangent
problem)) with every tangent system solved by sparse LU takes tens of
minutes per slab at full size (48x48x12 Q1 and 24x24x6 Q2, 86,436 free
DoFs each), so its final displacement is computed once by this script and
stored as ``newton_truth_<workload>.npz`` beside it:

* ``d``: the displacement at the last load level (free DoFs, FP64), Newton
  stopped at ||F|| <= 1e-11 ||F(d^{n,0})|| in every load step;
* ``digest``: SHA-256 of the workload's inputs (mesh, boundary sets,
  partition, fibres, material, loads), so that a test can tell whether the
  stored solution still belongs to the current input generators;
* ``log``: the oracle's per-Newton-step record (JSON).

Only ``oracle/`` and ``workloads/`` are used here; nothing comes from the
CUDA library.  Run ``python tests/golden/newton_truth.py [workload ...]``
from the repository root to regenerate.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
WORKLOADS = ("slab48_q1", "slab24_q2")
NEWTON_TOL = 1e-11


def input_digest(prob):
    """SHA-256 over the arrays and constants that define a workload."""
    h = hashlib.sha256()
    for key in ("elem_type", "coords", "elems", "elem_part", "n_parts", "dirichlet_nodes",
                "pressure_faces", "pressure", "gamma", "load_steps"):
        v = prob[key]
        if isinstance(v, str):
            h.update(v.encode())
        else:
            a = np.ascontiguousarray(np.asarray(v))
            h.update(str(a.dtype.kind).encode())
            h.update(str(a.shape).encode())
            h.update(a.astype(np.float64 if a.dtype.kind == "f" else np.int64).tobytes())
    h.update(json.dumps(prob["fibers"], sort_keys=True, default=float).encode())
    h.update(json.dumps(prob["material"], sort_keys=True, default=float).encode())
    return h.hexdigest()


def truth_path(name):
    return os.path.join(HERE, "newton_truth_%s.npz" % name)


def load_truth(name):
    z = np.load(truth_path(name))
    return z["d"], str(z["digest"]), json.loads(str(z["log"]))


def main(names):
    sys.path.insert(0, ROOT)
    from oracle.newton import direct_solver, newton_solve
    from workloads import slab_config
    for name in names:
        prob = slab_config(name)
        t0 = time.time()
        d, log = newton_solve(prob, direct_solver, tol=NEWTON_TOL)
        np.savez_compressed(truth_path(name), d=d, digest=np.array(input_digest(prob)),
                            log=np.array(json.dumps(log)))
        print("%s: %d Newton steps, %.0f s" % (name, len(log), time.time() - t0), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
