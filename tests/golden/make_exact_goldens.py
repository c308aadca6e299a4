"""Writes exact_goldens.json: Algorithm 1 evaluated by the FP64 oracle on
states too large for a test to sweep on the fly.

  * the twelve N = 18 T-doped random Clifford states of the exact-enumeration
    workload (eta in {1, 4, 16} x n_T in {0, 8, 32, 64}, seeds 100 + i);
  * sixteen states of the uneven batched workload (N ~ U{8..16} T-doped
    states, seeds 4000 + i): the first two of every N from 9 to 16.

Every state is |0^N> after its gate list, applied by the oracle in FP64 and
rounded to complex64 (oracle.circuit_state): the same array the GPU tests
upload. The sweep over x is split into ranges run in spawned processes
(families are independent) and summed in x order by oracle.exact_finalize.
Only oracle/ and the seeded input generators are called.

    python tests/golden/make_exact_goldens.py [--workers K]

The N = 18 part takes about 30 core-minutes per state.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "exact_goldens.json")
EPS = 1e-6


def state_sha(psi) -> str:
    return hashlib.sha256(np.ascontiguousarray(psi, dtype=np.complex64).tobytes()).hexdigest()[:16]


def _range_job(args):
    N, gates, x0, x1 = args
    import oracle
    psi = oracle.circuit_state(N, gates)
    fam, cnt = oracle.exact_families(psi, x0, x1, EPS)
    return x0, fam, cnt


def states():
    from paper_2601_00761_gb300 import inputs
    out = []
    seen = {}
    for sp in inputs.workload_batched_specs(count=4096):
        if 9 <= sp["N"] <= 16 and seen.get(sp["N"], 0) < 2:
            seen[sp["N"]] = seen.get(sp["N"], 0) + 1
            out.append({"set": "batched", "N": sp["N"], "eta": sp["eta"], "n_t": sp["n_t"], "seed": sp["seed"],
                        "index": sp["seed"] - 4000, "gates": inputs.batched_gate_list(sp)})
    for sp in inputs.workload_n18_gate_lists():
        out.append({"set": "n18", "N": 18, "eta": sp["eta"], "n_t": sp["n_t"], "seed": sp["seed"],
                    "gates": sp["gates"]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    import oracle
    oracle.build()
    recs = []
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool:
        for st in states():
            t0 = time.time()
            N, d = st["N"], 1 << st["N"]
            chunk = max(1, d // (4 * a.workers))
            jobs = [(N, st["gates"], x0, min(d, x0 + chunk)) for x0 in range(0, d, chunk)]
            fam = np.zeros((d, 4))
            cnt = np.zeros(d, dtype=np.int64)
            for x0, f, c in pool.imap_unordered(_range_job, jobs):
                fam[x0:x0 + len(c)] = f
                cnt[x0:x0 + len(c)] = c
            r = oracle.exact_finalize(fam, cnt, N)
            psi = oracle.circuit_state(N, st["gates"])
            rec = {k: st[k] for k in ("set", "N", "eta", "n_t", "seed")}
            if "index" in st:
                rec["index"] = st["index"]
            rec.update({"state_sha256_16": state_sha(psi), "M": [float(v) for v in r["M"]],
                        "S": [float(v) for v in r["S"]], "stab_count": int(r["stab_count"]),
                        "nullity": int(r["nullity"]), "eps_null": EPS})
            recs.append(rec)
            print(f"{st['set']} N={N} eta={st['eta']} n_t={st['n_t']}: M={rec['M']} nullity={rec['nullity']} "
                  f"({time.time() - t0:.0f}s)", flush=True)
            with open(OUT + ".tmp", "w") as f:
                json.dump({"_about": "Algorithm 1 by the FP64 oracle (oracle/sre_oracle.c) on complex64 "
                                     "states from oracle.circuit_state; written by make_exact_goldens.py",
                           "states": recs}, f, indent=1)
    os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
