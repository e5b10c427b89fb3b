"""Sensitivity of the oracle's pins (CPU, no GPU).

Each entry below plants one plausible mistake -- a wrong sign, a transposed
operand, a dropped term or factor, a wrong index, a missing slack -- in a
copy of the oracle's C source, builds that copy on its own, and runs
tests/test_oracle_pins.py against it (through NDG_ORACLE_LIB).  Every
mutant has to fail at least one pin; the unmodified source, built the same
way, has to pass.  The oracle in the repository is never modified.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ndg_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the mistake is, the passage it breaks, original text, planted text)
MUTATIONS = [
    ("children lose the radius floor", "Section 3.3 (R7)",
     "  if (g >= n_parents && child_k_min > 0.0 && child_k_min > r) r = child_k_min;",
     ""),
    ("radius floor applied to parents instead of children", "Section 3.3 (R7)",
     "  if (g >= n_parents && child_k_min > 0.0 && child_k_min > r) r = child_k_min;",
     "  if (g < n_parents && child_k_min > 0.0 && child_k_min > r) r = child_k_min;"),
    ("off-diagonal activation 2 sig - 1 -> sig - 1", "Eq. 2",
     "else if (j < i) v = 2.0 / (1.0 + exp(-th[PIDX(i, j)])) - 1.0;",
     "else if (j < i) v = 1.0 / (1.0 + exp(-th[PIDX(i, j)])) - 1.0;"),
    ("forward substitution divides -> multiplies by L_ii", "Eq. 1",
     "    z[i] = r / L[i * N + i];",
     "    z[i] = r * L[i * N + i];"),
    ("forward substitution uses L transposed", "Eq. 1",
     "    for (int j = 0; j < i; ++j) r -= L[i * N + j] * z[j];",
     "    for (int j = 0; j < i; ++j) r -= L[j * N + i] * z[j];"),
    ("exponent -s/2 -> -s", "Eq. 1",
     "      double ex = exp(-0.5 * s);\n      for (int k = 0; k < 3; ++k) acc[k]",
     "      double ex = exp(-s);\n      for (int k = 0; k < 3; ++k) acc[k]"),
    ("child mean L_p m_u + m_p -> L_p m_u - m_p", "Eq. 7",
     "      m[e * N + i] = s + mean[(size_t)g * N + i];",
     "      m[e * N + i] = s - mean[(size_t)g * N + i];"),
    ("child factor L_p U -> L_p U^T", "Eq. 6",
     "        for (int k = 0; k < N; ++k) s += Lp[i * N + k] * U[k * N + j];\n        Lc[i * N + j] = s;",
     "        for (int k = 0; k < N; ++k) s += Lp[i * N + k] * U[j * N + k];\n        Lc[i * N + j] = s;"),
    ("gradient w.r.t. the mean: wrong sign", "Section 4.1",
     "          gm[i] += h * (-2.0 * u[i]);",
     "          gm[i] += h * (2.0 * u[i]);"),
    ("gradient: back substitution with L instead of L^T", "Section 4.1",
     "          for (int j = i + 1; j < N; ++j) r -= Le[j * N + i] * u[j];",
     "          for (int j = i + 1; j < N; ++j) r -= Le[i * N + j] * u[j];"),
    ("gradient w.r.t. the weights: exp(-s/2) dropped", "Section 4.1",
     "          gw[c] += gb[c] * ex;",
     "          gw[c] += gb[c];"),
    ("off-diagonal activation derivative: factor 2 dropped", "Eq. 2",
     "        double dact = (j == i) ? exp(th) : 2.0 * sigm(th) * (1.0 - sigm(th));",
     "        double dact = (j == i) ? exp(th) : sigm(th) * (1.0 - sigm(th));"),
    ("colour gradient: brightness factor dropped", "Eq. 8",
     "      g_color[(size_t)g * 3 + k] = Gw[(size_t)g * 3 + k] * ap * sg * (1.0 - sg);",
     "      g_color[(size_t)g * 3 + k] = Gw[(size_t)g * 3 + k] * sg * (1.0 - sg);"),
    ("child chain: mean term of dL_p dropped", "Eq. 6-7",
     "          gLp[i * N + j] += s + gmc[i] * mu[j];",
     "          gLp[i * N + j] += s;"),
    ("child brightness gradient: alpha factor dropped", "Eq. 8",
     "        ga += Gw[c * 3 + k] * ac * sg;",
     "        ga += Gw[c * 3 + k] * sg;"),
    ("exact cull: sigma_r from L instead of L^T", "Eq. 4-5",
     "          for (int i = 0; i < N; ++i) tc += Lg[i * N + c] * r[i];",
     "          for (int i = 0; i < N; ++i) tc += Lg[c * N + i] * r[i];"),
    ("bucket contract: sigma_r from L instead of L^T", "Eq. 4-5",
     "        for (int i = c; i < N; ++i) tc = fmaf(Lf[i * N + c], r[i], tc);",
     "        for (int i = c; i < N; ++i) tc = fmaf(Lf[c * N + i], r[i], tc);"),
    ("bucket contract: lower slack bucket missing", "Section 3.2",
     "      int blo = bucket_raw(mr - ks, lo[j], ih[j], B) - 1;",
     "      int blo = bucket_raw(mr - ks, lo[j], ih[j], B);"),
    ("bucket contract: tile selection ignored", "Section 3.2",
     "      const long long t = sel ? sel[i] : i;",
     "      const long long t = i;"),
    ("cull radius sqrt(2 ln(w/c)) -> sqrt(ln(w/c))", "Eq. 5",
     "  return sqrt(2.0 * log(wm / cutoff));",
     "  return sqrt(log(wm / cutoff));"),
    ("conditioning: conditional mean shifted the wrong way", "Section 3.2",
     "      mu[(size_t)g * 3 + i] = mg[i] - z[i];",
     "      mu[(size_t)g * 3 + i] = mg[i] + z[i];"),
    ("conditioning: Schur-complement term of the weight with the wrong sign", "Section 3.2",
     "    for (int i = 0; i < 3; ++i) qc -= b[i] * z[i];",
     "    for (int i = 0; i < 3; ++i) qc += b[i] * z[i];"),
    ("conditioning: triangular solve with C transposed", "Section 3.2",
     "      for (int k = 0; k < i; ++k) s -= C[i * 3 + k] * y3[k];",
     "      for (int k = 0; k < i; ++k) s -= C[k * 3 + i] * y3[k];"),
    ("conditioned cull: sigma_r from T^T instead of T", "Section 3.2",
     "          for (int c = 0; c <= i; ++c) tc = fmaf(Lf[i * 3 + c], r[c], tc);",
     "          for (int c = 0; c <= i; ++c) tc = fmaf(Lf[c * 3 + i], r[c], tc);"),
    ("L2 loss gradient: factor 2 dropped", "Section 4.1",
     "    if (gbar) gbar[i] = 2.0 * d / n;",
     "    if (gbar) gbar[i] = d / n;"),
    ("relative L2: denominator from the target", "Section 4.1",
     "    double den = y[i] * y[i] + eps;",
     "    double den = target[i] * target[i] + eps;"),
    ("relative L2 gradient: denominator dropped", "Section 4.1",
     "    if (gbar) gbar[i] = 2.0 * d / den / n;",
     "    if (gbar) gbar[i] = 2.0 * d / n;"),
    ("Adam: first-moment bias correction dropped", "Adam",
     "    double mh = m1[i] / c1, vh = m2[i] / c2;",
     "    double mh = m1[i], vh = m2[i] / c2;"),
    ("densify: materialised mean L_p m_u - m_p", "Section 3.3",
     "      mean[(size_t)d * N + i] = s + mean[(size_t)g * N + i];",
     "      mean[(size_t)d * N + i] = s - mean[(size_t)g * N + i];"),
    ("densify: capacity exceeded by one", "Section 3.3",
     "  int room = G_cap - G, nflag = 0;",
     "  int room = G_cap - G + 1, nflag = 0;"),
    ("raw off-diagonal from L: inverse activation with the wrong sign", "Eq. 2",
     "          th = log((1.0 + lc) / (1.0 - lc));",
     "          th = log((1.0 - lc) / (1.0 + lc));"),
]


def _pins_pass(lib: str) -> bool:
    env = dict(os.environ, NDG_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode == 0


def test_every_planted_mistake_fails_a_pin(tmp_path):
    import oracle

    src = open(SRC).read()
    variants = [("unmodified source", src)]
    for what, _, orig, mut in MUTATIONS:
        assert src.count(orig) == 1, f"mutation site not unique or gone: {what}"
        variants.append((what, src.replace(orig, mut, 1)))

    def run(i):
        c = tmp_path / f"variant{i}.c"
        c.write_text(variants[i][1])
        lib = oracle.compile_source(str(c), str(tmp_path / f"variant{i}.so"))
        return _pins_pass(lib)

    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        passed = list(ex.map(run, range(len(variants))))
    assert passed[0], "the unmodified oracle, built the same way, fails its pins"
    missed = [variants[i][0] for i in range(1, len(variants)) if passed[i]]
    assert not missed, f"planted mistakes no pin catches: {missed}"
