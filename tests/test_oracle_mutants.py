"""The pins must catch plausible mistakes in the oracle.

Each mutant is a copy of talp_oracle.c with one planted error (a dropped
term, a wrong sign, a wrong index, a transposed operand, a missing clip),
compiled on the CPU into a temporary library; at least one pin of
test_oracle_pins must fail against it.
"""
import os

import pytest

import oracle
from test_oracle_pins import ALL_PINS

MUTANTS = [
    ("mpi_pe drops offload (Eq. 7)", "dout[1] = ratio_k(sU + sW, E,", "dout[1] = ratio_k(sU, E,"),
    ("host LB/CE use useful only", "maxUW = max64(maxUW, U + W);", "maxUW = max64(maxUW, U);"),
    ("elapsed drops MPI (Eq. 1)", "E = max64(E, U + W + P);\n        sU += U;", "E = max64(E, U + W);\n        sU += U;"),
    ("OE_host counts MPI (Eq. 8)", "dout[4] = ratio(sU, sU + sW);", "dout[4] = ratio(sU, sU + sW + sMPI);"),
    ("transfers not reduced by kernels", "int64_t DM = B - K;", "int64_t DM = UM;"),
    ("transfer sign flipped", "int64_t DM = B - K;", "int64_t DM = K - B;"),
    ("device OE uses device span (Eq. 12)", "dout[8] = ratio(maxB, E);", "dout[8] = ratio(maxB, maxB);"),
    ("CE_dev transposed (Eq. 11)", "dout[7] = ratio(maxK, maxB);", "dout[7] = ratio(maxB, maxK);"),
    ("LB_dev divides by n (Eq. 10)", "dout[6] = ratio_k(sK, (int64_t)m, maxK);",
     "dout[6] = ratio_k(sK, (int64_t)n_ranks, maxK);"),
    ("PE_dev divides by n (Eq. 9)", "dout[5] = ratio_k(sK, E, (int64_t)m);", "dout[5] = ratio_k(sK, E, (int64_t)n_ranks);"),
    ("max busy is max kernel + max transfer", "maxB = max64(maxB, K + DM);", "maxB = max64(maxB, K) + 0 * DM;"),
    ("device start not clipped", "int64_t s = max64(dev_se[2 * j], a);\n                int64_t e = min64(dev_se[2 * j + 1], b);\n                if (e <= s) continue;\n                ivl_t x",
     "int64_t s = dev_se[2 * j];\n                int64_t e = min64(dev_se[2 * j + 1], b);\n                if (e <= s) continue;\n                ivl_t x"),
    ("concurrency start not clipped", "int64_t s = max64(dev_se[2 * j], a);\n                int64_t e = min64(dev_se[2 * j + 1], b);\n                if (e <= s) continue;\n                ea[na]",
     "int64_t s = dev_se[2 * j];\n                int64_t e = min64(dev_se[2 * j + 1], b);\n                if (e <= s) continue;\n                ea[na]"),
    ("host end not clipped", "int64_t hi = min64(host_se[2 * j + 1], b);", "int64_t hi = host_se[2 * j + 1];"),
    ("kind read from the stream bits", "if ((dev_tag[j] >> 5) == 0) kv", "if ((dev_tag[j] & 31) == 0) kv"),
    ("nested interval shrinks the run", "} else if (v[j].e > ce) {   /* overlapping or touching: extend */",
     "} else {   /* overlapping or touching: extend */"),
    ("union drops the last run", "    total += ce - cs;\n    return total;", "    return total;"),
    ("host state collapsed", "if (hi > lo) acc[host_state[j]] += hi - lo;", "if (hi > lo) acc[0] += hi - lo;"),
    ("idle uses window start", "sIdle += len - B;", "sIdle += win[2 * i] - B;"),
    ("hidden transfer sign", "sHidden += K + UM - B;", "sHidden += K - UM + B;"),
    ("0/0 reads as 0", "if (k == 0 || den == 0) return 1.0;", "if (k == 0 || den == 0) return 0.0;"),
    ("validation ignores kind", "if ((dev_tag[j] >> 5) > 4) bad |= 8;", "if ((dev_tag[j] >> 5) > 7) bad |= 8;"),
    ("concurrency levels off by one", "for (int64_t k = 1; k <= c && k <= (int64_t)K; ++k)",
     "for (int64_t k = 1; k < c && k <= (int64_t)K; ++k)"),
    ("concurrency end not clipped", "                int64_t e = min64(dev_se[2 * j + 1], b);\n                if (e <= s) continue;\n                ea[na]",
     "                int64_t e = dev_se[2 * j + 1];\n                if (e <= s) continue;\n                ea[na]"),
    ("strong scalability inverted", "o[1] = weak ? ratio_scaled(U0, n, U, n0) : ratio(U0, U);",
     "o[1] = weak ? ratio_scaled(U0, n, U, n0) : ratio(U, U0);"),
    ("weak scalability uses the reference's ranks twice", "o[3] = weak ? ratio_scaled(K0, m, Kd, m0) : ratio(K0, Kd);",
     "o[3] = weak ? ratio_scaled(K0, m0, Kd, m0) : ratio(K0, Kd);"),
    ("global efficiency of the reference run", "o[2] = pe[2 * r] * o[1];", "o[2] = pe[2 * ref] * o[1];"),
    ("concurrency kernels read from stream bits", "if ((dev_tag[j] >> 5) == 0) {\n                    ek[nk]",
     "if ((dev_tag[j] & 31) == 0) {\n                    ek[nk]"),
    ("thread tree: processes not weighted by their threads", "sTM += T * M;", "sTM += M;"),
    ("thread tree: the master stands for its process", "M = max64(M, U + W);",
     "if (u == proc_off[i]) M = U + W;"),
    ("thread tree: elapsed over masters only", "E = max64(E, U + W + P);\n            sU += U;",
     "if (u == proc_off[i]) E = max64(E, U + W + P);\n            sU += U;"),
    ("thread tree: OE over the busiest threads", "dout[5] = ratio(sU, sU + sW);", "dout[5] = ratio(sU, sTM);"),
    ("thread tree: offload not busy", "M = max64(M, U + W);", "M = max64(M, U);"),
    ("thread tree: thread LB over the largest busiest thread", "dout[4] = ratio(sU + sW, sTM);",
     "dout[4] = ratio(sU + sW, nT * maxM);"),
    ("thread tree: nT counts processes", "nT += T;", "nT += 1;"),
    ("thread tree: MPI CE transposed", "dout[3] = ratio(maxM, E);", "dout[3] = ratio(E, maxM);"),
    ("thread tree: next process starts one unit late", "for (uint32_t u = proc_off[i]; u < proc_off[i + 1]; ++u)",
     "for (uint32_t u = proc_off[i] + (i > 0); u < proc_off[i + 1]; ++u)"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation site not unique/present: {old!r}"
    mut = os.path.join(tmp_path, "mutant.c")
    open(mut, "w").write(src.replace(old, new))
    lib = oracle.compile_c(mut, os.path.join(tmp_path, "libmutant.so"))
    O = oracle.Oracle(lib)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(O)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin catches mutant: {name}"
