"""The oracle's pins catch plausible mistakes: each mutant below plants one
(a wrong constant, sign, index, weight, class, bound or dropped term, or a
slip in the epoch logic of Alg. 4 or in App. E's score) in a copy of
oracle/gcp_oracle.c, oracle/driver.py or oracle/score.py, on the CPU, and the oracle's pin tests
(tests/test_oracle_*.py, tests/test_paper_facts.py) must fail on it.  The
product library is not involved.  A mutant whose site is no longer in the
source fails this test too, so the list follows the oracle as it changes.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, the text it changes (first occurrence), the mistaken text)
MUTANTS = [
    ('philox M0 bit',
     '0xD2E7470EE14C6C93ULL',
     '0xD2E7470EE14C6C92ULL'),
    ('philox key bump from round 2',
     'if (round > 0) { k0 += W0; k1 += W1; }',
     'if (round > 1) { k0 += W0; k1 += W1; }'),
    ('philox n0 uses c3',
     'uint64_t n0 = hi1 ^ c1 ^ k0;',
     'uint64_t n0 = hi1 ^ c3 ^ k0;'),
    ('philox 9 rounds',
     'round < 10',
     'round < 9'),
    ('randi low word',
     '    mul128(word, n, &hi, &lo);\n    return hi;',
     '    mul128(word, n, &hi, &lo);\n    return lo % n;'),
    ('block per 2 modes',
     '(uint64_t)(k / 4)};',
     '(uint64_t)(k / 2)};'),
    ('word shift',
     'idx[k] = (int64_t)orc_randi(w[k % 4]',
     'idx[k] = (int64_t)orc_randi(w[(k + 1) % 4]'),
    ('counter j/stream swapped',
     'uint64_t ctr[4] = {j, stream, (uint64_t)tag, (uint64_t)(k / 4)};',
     'uint64_t ctr[4] = {stream, j, (uint64_t)tag, (uint64_t)(k / 4)};'),
    ('nonzero word 1',
     'return (int64_t)orc_randi(w[0], (uint64_t)nnz);',
     'return (int64_t)orc_randi(w[1], (uint64_t)nnz);'),
    ('nonzero tag uniform',
     'uint64_t ctr[4] = {j, stream, (uint64_t)ORC_TAG_NONZERO, 0};',
     'uint64_t ctr[4] = {j, stream, (uint64_t)ORC_TAG_UNIFORM, 0};'),
    ('linear key reversed strides',
     'key = key * (uint64_t)dims[k] + (uint64_t)idx[k];',
     'key = key * (uint64_t)dims[d - 1 - k] + (uint64_t)idx[k];'),
    ('odds f sign',
     'return log(mp + 1.0) - x * log(mp);',
     'return log(mp + 1.0) + x * log(mp);'),
    ('identity g',
     'return 1.0 - x / mp;',
     'return 1.0 - x / (mp * mp);'),
    ('gamma f sign',
     'return x / mp + log(mp);',
     'return x / mp - log(mp);'),
    ('beta f factor',
     'return 2.0 * sqrt(mp) + 2.0 * x / sqrt(mp);',
     'return 2.0 * sqrt(mp) + x / sqrt(mp);'),
    ('gaussian g no 2',
     'return 2.0 * (m - x);',
     'return (m - x);'),
    ('gaussian f half',
     'return (x - m) * (x - m);',
     'return 0.5 * (x - m) * (x - m);'),
    ('logit f sign',
     'return softplus - x * m;',
     'return softplus + x * m;'),
    ('logit g sign',
     'return sig - x;',
     'return sig + x;'),
    ('poisson f',
     'return exp(m) - x * m;',
     'return exp(m) - x * exp(m);'),
    ('beta g',
     'return 1.0 / sqrt(mp) - x / (mp * sqrt(mp));',
     'return 1.0 / sqrt(mp) - x / (2.0 * mp * sqrt(mp));'),
    ('odds g',
     'return 1.0 / (mp + 1.0) - x / mp;',
     'return 1.0 / (mp + 1.0) - x / (mp + 1.0);'),
    ('gamma g',
     'return -x / (mp * mp) + 1.0 / mp;',
     'return -x / (mp * mp) - 1.0 / mp;'),
    ('model column 0',
     'for (int k = 0; k < d; ++k) prod *= A[off[k] + idx[k] * rank + j];',
     'for (int k = 0; k < d; ++k) prod *= A[off[k] + idx[k] * rank + 0];'),
    ('mode offsets',
     'off[k] = off[k - 1] + dims[k - 1] * rank;',
     'off[k] = off[k - 1] + dims[k] * rank;'),
    ('membership any',
     '    return lo < nnz && sorted_keys[lo] == key;\n}',
     '    return lo < nnz && sorted_keys[lo] <= key + 1;\n}'),
    ('sparse value default 1',
     '? sorted_vals[lo] : 0.0;',
     '? sorted_vals[lo] : 1.0;'),
    ('uniform sparse weight',
     '                w_out[j] = omega / (double)q;\n',
     '                w_out[j] = 1.0 / (double)q;\n'),
    ('uniform dense weight v dropped',
     '(omega / (double)q) * (dense_weights ? dense_weights[key] : 1.0);',
     '(omega / (double)q);'),
    ('observed weight omega',
     'w_out[accepted] = (observed / (double)q) * dense_weights[key];',
     'w_out[accepted] = (omega / (double)q) * dense_weights[key];'),
    ('observed accept negative only',
     'if (dense_weights[key] == 0.0) continue;',
     'if (dense_weights[key] < 0.0) continue;'),
    ('observed v dropped',
     'w_out[accepted] = (observed / (double)q) * dense_weights[key];',
     'w_out[accepted] = (observed / (double)q);'),
    ('nonzero weight omega',
     'w_out[j] = eta / (double)p;',
     'w_out[j] = omega / (double)p;'),
    ('binary value 0',
     'x_out[j] = coo_vals ? coo_vals[xi] : 1.0;',
     'x_out[j] = coo_vals ? coo_vals[xi] : 0.0;'),
    ('semi zero weight zeta',
     'w_out[p + j] = omega / (double)q;',
     'w_out[p + j] = (omega - eta) / (double)q;'),
    ('strat zero weight omega',
     'w_out[pos] = zeta / (double)q;',
     'w_out[pos] = omega / (double)q;'),
    ('strat rho ignored',
     'int64_t batch = q > 0 ? (int64_t)ceil(rho * (double)q * omega / zeta) : 0;',
     'int64_t batch = q > 0 ? (int64_t)ceil((double)q * omega / zeta) : 0;'),
    ('strat cap 65',
     '    int64_t cap = 64 * batch;\n    int64_t accepted = 0, c = 0;\n    int64_t ix[ORC_MAX_D];\n    while (accepted < q) {\n        if (c >= cap) {\n            if (candidates_used) *candidates_used = c;\n            return ORC_ERR_SHORTFALL;\n        }\n        orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_ZERO_CANDIDATE',
     '    int64_t cap = 65 * batch;\n    int64_t accepted = 0, c = 0;\n    int64_t ix[ORC_MAX_D];\n    while (accepted < q) {\n        if (c >= cap) {\n            if (candidates_used) *candidates_used = c;\n            return ORC_ERR_SHORTFALL;\n        }\n        orc_draw_multi_index(d, dims, seed, problem, stream, ORC_TAG_ZERO_CANDIDATE'),
    ('semi class strat',
     'cls_out[j] = kind == ORC_STRATIFIED ? ORC_CLS_STRAT_NZ : ORC_CLS_SEMI_NZ;',
     'cls_out[j] = ORC_CLS_STRAT_NZ;'),
    ('semi y no g0',
     'if (cls == ORC_CLS_SEMI_NZ) return w * (orc_loss_g(loss, x, m) - orc_loss_g(loss, 0.0, m));',
     'if (cls == ORC_CLS_SEMI_NZ) return w * orc_loss_g(loss, x, m);'),
    ('semi f plus',
     'w * (orc_loss_f(loss, x, m) - orc_loss_f(loss, 0.0, m))',
     'w * (orc_loss_f(loss, x, m) + orc_loss_f(loss, 0.0, m))'),
    ('grad skips mode 0 in products',
     '                    if (l != k) prod *= A[off[l] + ix[l] * rank + j];\n                G[off[k] + ix[k] * rank + j] += y * prod;',
     '                    if (l != k && l != 0) prod *= A[off[l] + ix[l] * rank + j];\n                G[off[k] + ix[k] * rank + j] += y * prod;'),
    ('grad half',
     '                G[off[k] + ix[k] * rank + j] += y * prod;\n            }\n        }\n    }\n    return ORC_OK;',
     '                G[off[k] + ix[k] * rank + j] += 0.5 * y * prod;\n            }\n        }\n    }\n    return ORC_OK;'),
    ('full grad weight dropped',
     'double wt = v ? v[lin] : 1.0;',
     'double wt = 1.0;'),
    ('full F weight dropped',
     'F += wt * orc_loss_f(loss, X[lin], m);',
     'F += orc_loss_f(loss, X[lin], m);'),
    ('full grad column-major decode',
     'for (int k = d - 1; k >= 0; --k) { ix[k] = rem % dims[k]; rem /= dims[k]; }',
     'for (int k = 0; k < d; ++k) { ix[k] = rem % dims[k]; rem /= dims[k]; }'),
    ('adam bias power t+2',
     'double c1 = 1.0 - pow(beta1, (double)(t + 1));',
     'double c1 = 1.0 - pow(beta1, (double)(t + 2));'),
    ('adam c2 power t+2',
     'double c2 = 1.0 - pow(beta2, (double)(t + 1));',
     'double c2 = 1.0 - pow(beta2, (double)(t + 2));'),
    ('adam C abs',
     'C[e] = beta2 * C[e] + (1.0 - beta2) * G[e] * G[e];',
     'C[e] = beta2 * C[e] + (1.0 - beta2) * fabs(G[e]);'),
    ('adam eps swapped',
     'double den = eps_inside_sqrt ? sqrt(ch + eps) : sqrt(ch) + eps;',
     'double den = eps_inside_sqrt ? sqrt(ch) + eps : sqrt(ch + eps);'),
    ('adam projection to 0',
     'if (A[e] < lower) A[e] = lower;',
     'if (A[e] < lower) A[e] = 0.0;'),
    ('adam no bias correction B',
     'double bh = B[e] / c1;',
     'double bh = B[e];'),
    ('adam B uses beta2',
     'B[e] = beta1 * B[e] + (1.0 - beta1) * G[e];',
     'B[e] = beta1 * B[e] + (1.0 - beta2) * G[e];'),
    ('estimate weight dropped',
     'F += orc_entry_f(loss, cls[e], x[e], m, w[e]);',
     'F += orc_entry_f(loss, cls[e], x[e], m, 1.0);'),
    ('count observed',
     'if (weights[i] != 0.0) c++;',
     'if (weights[i] > 0.5) c++;'),
    ('grad abs drops fabs',
     'Gabs[off[k] + ix[k] * rank + j] += fabs(y * prod);',
     'Gabs[off[k] + ix[k] * rank + j] += y * prod;'),
    ('loss abs drops fabs',
     'S += fabs(orc_entry_f(loss, cls[e], x[e], m, w[e]));',
     'S += orc_entry_f(loss, cls[e], x[e], m, w[e]);'),
    ('M_EPS 1e-3',
     '#define ORC_M_EPS 1e-10',
     '#define ORC_M_EPS 1e-3'),
    ('observed cap 65 batches',
     'int64_t cap = 64 * batch;',
     'int64_t cap = 65 * batch;'),
]

# the same for the Alg. 4 loop of oracle/driver.py
DRIVER_MUTANTS = [
    ('failed epoch keeps its moments', '            A, B, C = saved\n', '            A, _, _ = saved\n'),
    ('failed epoch keeps its factors', '            A, B, C = saved\n', '            _, B, C = saved\n'),
    ('t not wound back', '            t -= tau\n', '            t -= 0\n'),
    ('stream wound back', '            t -= tau\n', '            t -= tau\n            it -= tau\n'),
    ('alpha not decayed', '            alpha *= nu\n', '            alpha *= 1.0\n'),
    ('equal estimate rejected', 'if not (F <= F_old):', 'if not (F < F_old):'),
    ('one failure too many allowed', 'while c <= kappa and', 'while c <= kappa + 1 and'),
    ('estimate not restored', '            F = F_old\n', '            pass\n'),
    ('stream per epoch instead of per iteration', '            it += 1\n', '            it += 0\n'),
]

# and for App. E's cosine score of oracle/score.py
SCORE_MUTANTS = [
    ('score not averaged over components', 'return float(best / r)', 'return float(best)'),
    ('estimate columns not normalised', 'bn = b / np.linalg.norm(b, axis=0, keepdims=True)', 'bn = b'),
    ('assignment minimises instead of maximising', 'linear_sum_assignment(-prod)', 'linear_sum_assignment(prod)'),
]


def pin_tests():
    tests = sorted(f for f in os.listdir(os.path.join(ROOT, "tests")) if f.startswith("test_oracle_"))
    return [os.path.join("tests", f) for f in tests] + [os.path.join("tests", "test_paper_facts.py")]


def run_mutant(workdir, rel, src, mutant):
    name, old, new = mutant
    d = os.path.join(workdir, name.replace(" ", "_").replace("/", "_"))
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"), ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(d, "paper_1906_01687_gb300"))
    for f in ("__init__.py", "synth.py"):  # the seeded input generators some pins use
        shutil.copy(os.path.join(ROOT, "paper_1906_01687_gb300", f), os.path.join(d, "paper_1906_01687_gb300", f))
    with open(os.path.join(d, rel), "w") as f:
        f.write(src.replace(old, new, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pin_tests()],
                       cwd=d, capture_output=True, text=True, timeout=600)
    return name, r.returncode


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    jobs = []
    for rel, mutants in ((os.path.join("oracle", "gcp_oracle.c"), MUTANTS),
                         (os.path.join("oracle", "driver.py"), DRIVER_MUTANTS),
                         (os.path.join("oracle", "score.py"), SCORE_MUTANTS)):
        with open(os.path.join(ROOT, rel)) as f:
            src = f.read()
        missing = [m[0] for m in mutants if m[1] not in src]
        assert not missing, f"mutation sites no longer in {rel}: {missing}"
        jobs += [(rel, src, m) for m in mutants]
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda job: run_mutant(str(tmp_path), *job), jobs))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"mistakes no pin catches: {survivors}"
