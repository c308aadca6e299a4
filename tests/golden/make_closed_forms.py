"""Writes closed_forms.json: values the paper prints or derives in closed
form, each with its citation. Evaluates the paper's formulas only (plain
Python math); it calls neither the oracle nor the CUDA path.

    python tests/golden/make_closed_forms.py
"""
import json
import math
import os

out = {"_about": "closed forms from Xiao & Ryu, arXiv 2601.00761; logs base 2",
       "t_product_state": [], "psi_m_family_m2": [], "haar": []}

# |T>^k (x) |0>^(N-k): per-qubit Pauli weights (SM Sec. II A: |<T|I|T>|^4 +
# |<T|Z|T>|^4 = 1, |<T|X|T>|^4 + |<T|Y|T>|^4 = 1/2) give M_2 = k log2(4/3)
# (main text, "Clifford preconditioning"); the same single-qubit expectations
# (c_I = 1, c_X = c_Y = 1/sqrt2, c_Z = 0) give M_1 = k/2 and
# M_3 = (k/2) log2(8/5); the stabilizer group of |T> is {I}, so nu = k.
for N in range(1, 9):
    for k in range(0, N + 1):
        out["t_product_state"].append({
            "N": N, "k": k, "M1": k / 2.0, "M2": k * math.log2(4.0 / 3.0),
            "M3": (k / 2.0) * math.log2(8.0 / 5.0), "nullity": k,
            "cite": "main text (M2 = N_T log2(4/3)); SM Sec. II A per-qubit moments"})

# |psi_m> = |T>^{N/2} |0>^{N/2}, even N: m_{2;x} = 2^{-3N/2-k} when x_B = 0
# and wt(x_A) = k, else 0 (SM Eq. S4); E_x[m_{2;x}] = (3/64)^{N/2} (SM Eq. S5);
# r_2 exact (SM Eq. S6).  The T qubits are qubits 0..N/2-1 (low bits of x).
for N in (2, 4, 6, 8):
    h = N // 2
    fam = []
    for x in range(1 << N):
        xA, xB = x & ((1 << h) - 1), x >> h
        fam.append(0.0 if xB else 2.0 ** (-1.5 * N - bin(xA).count("1")))
    Ex = (3.0 / 64.0) ** h
    r2 = (8.0 / 3.0) ** h * math.sqrt(
        ((5.0 / 4.0) ** h - 1.0) / (4.0 ** h - 1.0)
        - ((1.5 ** h - 1.0) ** 2) / (4.0 ** h - 1.0) ** 2)
    out["psi_m_family_m2"].append({"N": N, "m2_x": fam, "E_x": Ex, "r2": r2,
                                   "cite": "SM Eqs. S4, S5, S6"})

# Haar: E[(1/d) sum_P c_P^4] = 4/(d+3), M2_Haar = log2(d+3) - 2 (main text,
# "Monte Carlo sampling with FWHT"; SM Eq. Mlin_multi long-time limit).
# The paper's MC value at N=24 with 10 sampled x: 21.9999(2).
for N in range(1, 31):
    d = 2 ** N
    out["haar"].append({"N": N, "E_sum_c4_over_d": 4.0 / (d + 3.0),
                        "M2_haar": math.log2(d + 3.0) - 2.0})
out["haar_paper_mc_N24"] = {"M2": 21.9999, "err": 0.0002, "n_x": 10,
                            "cite": "main text, Monte Carlo section (Haar example)"}

path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
with open(path, "w") as f:
    json.dump(out, f, indent=1)
print("wrote", path)
