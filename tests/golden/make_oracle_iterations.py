"""Write oracle_iterations_convdiff2d_1024.json: iterations the CPU oracle needs to reach
a 1e-10 true relative residual on the 1024x1024 convection-diffusion system (Jacobi,
FP64, periodic replacement every 100 iterations).  Calls only oracle/ and testproblems/.
Used by the full-size GPU test of the replacement schedule.  Takes a few minutes."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import testproblems as tp  # noqa: E402
from oracle import krylov  # noqa: E402

if __name__ == "__main__":
    p = tp.problem_convdiff2d(1024)
    A = p.A.to_scipy()
    out = {}
    for name, kw in [("fp64_rr100", dict(rr_period=100)), ("fp64_plain", dict())]:
        t = time.time()
        r = krylov.pbicgstab(A, p.b, precond="jacobi", tol=1e-10, maxit=20000, **kw)
        out[name] = dict(iterations=r.iterations, status=r.status.name, rel_res_true=r.rel_res_true,
                         n_replacements=r.n_replacements, seconds=round(time.time() - t, 1))
        print(name, out[name], flush=True)
    out["workload"] = "convdiff2d_1024x1024, Jacobi, tol 1e-10, x0 = 0 (testproblems.problem_convdiff2d(1024))"
    json.dump(out, open(os.path.join(HERE, "oracle_iterations_convdiff2d_1024.json"), "w"), indent=1)
