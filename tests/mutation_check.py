"""Mutation check of the oracle's pins (test infrastructure, not collected by pytest).

Each entry plants one plausible mistake in a copy of ``oracle/lbdps_oracle.c``
(a dropped term, a wrong sign, index, stride or constant, a branch limit moved),
builds the copy into a library of its own in a temporary folder under
``_build/``, and runs ``tests/test_oracle_pins.py`` against it
(``LBDPS_ORACLE_LIB`` makes the oracle load that library).  A mutant that passes every pin marks a part of the oracle
that the pins do not fix.  The committed source is never modified.

    python tests/mutation_check.py [-j JOBS] [-k SUBSTRING ...]

Exit status 0 when every mutant is caught.
"""
import argparse
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle import build as oracle_build  # noqa: E402

SRC = os.path.join(ROOT, "oracle", "lbdps_oracle.c")

# (name, text in the oracle source, the planted replacement)
MUTANTS = [
    # coupled step, hard spheres, soft spheres, friction, sequential rule, solids loop
    ('gamma_t swapped',
     '(1.0 / tau_t) * (1.0 - g_taut)',
     '(1.0 / tau_t) * (1.0 - g_tau)'),
    ('node at corner',
     'double t = p[a] - 0.5;',
     'double t = p[a];'),
    ('half force dropped',
     '+ 0.5 * b->k.fb[a]) /',
     ') /'),
    ('omega_s sign',
     'double omega_s = fi[io] - fi[i] + fe_s[i] - fe[io];',
     'double omega_s = fi[i] - fi[io] + fe_s[i] - fe[io];'),
    ('eps3d for gamma',
     'double g_tau = ob_gamma(b->eps_s[x], tau);',
     'double g_tau = ob_gamma(1.0 - b->eps_g[x], tau);'),
    ('guo prefactor',
     'src *= (1.0 - 0.5 / tau_t) * b->w[i];',
     'src *= b->w[i];'),
    ('outlet uses inlet',
     'for (int a = 0; a < dim; ++a) uin[a] = b->u[x * 3 + a];',
     'for (int a = 0; a < dim; ++a) uin[a] = 0.0;'),
    ('pressure factor',
     'gp = (b->rho[xh] - b->rho[xl]) / 3.0 / span;',
     'gp = (b->rho[xh] - b->rho[xl]) / 3.0;'),
    ('approach sign',
     'if (!(dot < 0.0)) continue;\n                if (b->id[p] < b->id[j])',
     'if (!(dot <= 0.0)) continue;\n                if (b->id[p] < b->id[j])'),
    ('min image',
     'if (d > 0.5 * L) d -= L;',
     'if (d > L) d -= L;'),
    ('restitution wall',
     'vnew[p * 3 + a] = -b->k.e * vnew[p * 3 + a];',
     'vnew[p * 3 + a] = -vnew[p * 3 + a];'),
    ('mirror',
     '*pa = -*pa;',
     '*pa = 0.0;'),
    ('beta slip uses u',
     'double sl = b->uact[x * 3 + a] - vs[a];',
     'double sl = b->u[x * 3 + a] - vs[a];'),
    ('les 18',
     '18.0 * cs * cs * qn / rho',
     '18.0 * cs * cs * qn'),
    ('scale abs',
     'scale = fabs(b->fpg[x * 3 + a]) / fabs(S[a]);',
     'scale = b->fpg[x * 3 + a] / fabs(S[a]);'),
    ('eq10 radius',
     'es = (double)n * M_PI * b->k.r * b->k.r;      /* Eq. 10, h = 1 */',
     'es = (double)n * M_PI * b->k.d * b->k.r;'),
    ('moving wall',
     'val - 6.0 * b->w[i] * b->rho[x] * cu',
     'val - 3.0 * b->w[i] * b->rho[x] * cu'),
    ('gravity eff',
     'k->g_eff[a] = (1.0 - s->rho_g / s->rho_s) * s->g[a] * gscale;',
     'k->g_eff[a] = s->g[a] * gscale;'),
    ('soft damping sign',
     'double f = kn * (d - dist) - b->k.eta * vn;',
     'double f = kn * (d - dist) + b->k.eta * vn;'),
    ('soft pair mass',
     'k->eta = 2.0 * z * sqrt(0.5 * k->mp * k->kn);',
     'k->eta = 2.0 * z * sqrt(k->mp * k->kn);'),
    ('soft no clip',
     'if (f < 0.0) f = 0.0;\n                /* contact point',
     '/* contact point'),
    ('soft wall dropped',
     'double f = kn * (r - l) - b->k.eta_w * (va * nrm[a]);',
     'double f = 0.0;'),
    ('soft force unused',
     'if (b->model == 1) fa += b->fc[p * 3 + a];',
     'if (b->model == 2) fa += b->fc[p * 3 + a];'),
    ('friction torque arm',
     'arm[a] = -l * nrm[a];',
     'arm[a] = l * nrm[a];'),
    ('friction lever',
     'double l = 0.5 * dist, ws[3]',
     'double l = b->k.r, ws[3]'),
    ('friction coulomb',
     'double mag = b->k.gamma_t * st, cap = b->k.mu_f * fn;',
     'double mag = b->k.gamma_t * st, cap = 2.0 * b->k.mu_f * fn;'),
    ('inertia',
     'k->inertia = 0.4 * k->mp * k->r * k->r;',
     'k->inertia = 0.5 * k->mp * k->r * k->r;'),
    ('seq recheck',
     '            if (!(dot < 0.0)) continue;\n            ob_binary_collision',
     '            ob_binary_collision'),
    ('recirc wrap',
     '                    *pa -= L;\n                    b->solids_out += 1;',
     '                    *pa = 0.0;\n                    b->solids_out += 1;'),
    ('recirc count',
     '                    b->solids_out += 1;',
     '                    b->solids_out += 2;'),
    # the 3D paths
    ('d3q19 weights',
     '(i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0)',
     '(i <= 6 ? 1.0 / 36.0 : 1.0 / 18.0)'),
    ('d3q19 velocities',
     '{0, 1, -1}, {0, -1, 1}};',
     '{1, 1, -1}, {-1, -1, 1}};'),
    ('stencil z stride',
     'nodes[k] = idx[0] + (int64_t)b->n[0] * (idx[1] + (int64_t)b->n[1] * idx[2]);',
     'nodes[k] = idx[0] + (int64_t)b->n[0] * (idx[1] + (int64_t)b->n[0] * idx[2]);'),
    ('gradp z stride',
     'int64_t stride = (a == 0) ? 1 : (a == 1) ? b->n[0] : (int64_t)b->n[0] * b->n[1];',
     'int64_t stride = (a == 0) ? 1 : (a == 1) ? b->n[0] : (int64_t)b->n[0] * b->n[0];'),
    ('eq11 in 3d',
     'return b->dim == 2 ? ob_eps3d(1.0 - es) : 1.0 - es;',
     'return ob_eps3d(1.0 - es);'),
    ('cap3d',
     'const double cap3d = M_PI / (3.0 * sqrt(2.0));',
     'const double cap3d = M_PI / (2.0 * sqrt(3.0));'),
    ('bubble 3d stride',
     'int64_t stride[3] = {1, b->n[0], (int64_t)b->n[0] * b->n[1]};\n    int vert = b->dim - 1;\n    out[0]',
     'int64_t stride[3] = {1, b->n[0], (int64_t)b->n[0] * b->n[0]};\n    int vert = b->dim - 1;\n    out[0]'),
    ('bubble vertical',
     'int vert = b->dim - 1;\n    out[0]',
     'int vert = 1;\n    out[0]'),
    ('3d inlet index',
     '(vert == 1) ? (x % b->n[0]) : (x % ((int64_t)b->n[0] * b->n[1]))',
     '(vert == 1) ? (x % b->n[0]) : (x % b->n[0])'),
    ('les dims',
     'for (int bb = 0; bb < dim; ++bb) {',
     'for (int bb = 0; bb < 2; ++bb) {'),
    ('cross3 sign',
     'c[1] = a[2] * b[0] - a[0] * b[2];',
     'c[1] = a[0] * b[2] - a[2] * b[0];'),
    ('3d spin update',
     'for (int a = 0; a < 3; ++a) b->spin[p * 3 + a] += b->tq[p * 3 + a] / b->k.inertia;',
     'for (int a = 2; a < 3; ++a) b->spin[p * 3 + a] += b->tq[p * 3 + a] / b->k.inertia;'),
    # the faces of the domain
    ('upper wall clamps',
     '*pa = 2.0 * L - *pa;',
     '*pa = nextafter(L, 0.0);'),
    ('upper wall elastic',
     '*pa = 2.0 * L - *pa;\n                        b->v[p * 3 + a] = -b->k.e * b->v[p * 3 + a];',
     '*pa = 2.0 * L - *pa;\n                        b->v[p * 3 + a] = -b->v[p * 3 + a];'),
    ('lower periodic mirrors',
     '*pa += L;\n                        if (*pa >= L) *pa = 0.0;',
     '*pa = -*pa;\n                        if (*pa >= L) *pa = 0.0;'),
    ('walls two axes',
     '/* specular walls and periodic wrap */\n            for (int a = 0; a < dim; ++a) {',
     '/* specular walls and periodic wrap */\n            for (int a = 0; a < 2; ++a) {'),
    ('eq16 two axes',
     'for (int a = 0; a < dim; ++a) {\n                double fa = b->fd',
     'for (int a = 0; a < 2; ++a) {\n                double fa = b->fd'),
    ('min image lower',
     'else if (d < -0.5 * L) d += L;',
     'else if (d < -0.5 * L) d -= L;'),
    ('one-sided span lo',
     'else { lo = idx[a]; span = 1.0; } }',
     'else { lo = idx[a]; span = 2.0; } }'),
    ('one-sided span hi',
     'else { hi = idx[a]; span = 1.0; } }',
     'else { hi = idx[a]; span = 2.0; } }'),
    ('stencil clamps periodic',
     'lo = (lo % b->n[a] + b->n[a]) % b->n[a];',
     'lo = lo < 0 ? 0 : lo;'),
    ('stencil wrap hi',
     'hi = (hi % b->n[a] + b->n[a]) % b->n[a];',
     'hi = hi >= b->n[a] ? b->n[a] - 1 : hi;'),
    # the step statistics
    ('slip cell mean',
     'ss += (double)b->ntot[x] * sqrt(sl);\n            nw += (double)b->ntot[x];',
     'ss += sqrt(sl);\n            nw += 1.0;'),
    ('slip uses u',
     'double d = b->uact[x * 3 + a] - b->vs[x * 3 + a];',
     'double d = b->u[x * 3 + a] - b->vs[x * 3 + a];'),
    ('momentum without mass',
     'nsum(&s[4 + a], &c[4 + a], b->k.mp * b->v[p * 3 + a]);',
     'nsum(&s[4 + a], &c[4 + a], b->v[p * 3 + a]);'),
    # the closure laws (Eq. 9, 19-22)
    ('gamma tau',
     'return eps_s * (tau - 0.5) / ((1.0 - eps_s) + (tau - 0.5));',
     'return eps_s * tau / ((1.0 - eps_s) + tau);'),
    ('omega b1 offset',
     '0.0214 / (4.0 * t * t + 0.0044) - 0.5760',
     '0.0214 / (4.0 * t * t + 0.0044) - 0.5670'),
    ('omega b2 centre',
     'double t = eps_g - 0.7789;',
     'double t = eps_g - 0.7798;'),
    ('omega b3 intercept',
     '32.8295 * eps_g - 31.8295',
     '32.8295 * eps_g - 31.8259'),
    ('omega b1 upper',
     'if (eps_g <= 0.82) {',
     'if (eps_g <= 0.85) {'),
    ('re exponent',
     'pow(re, 0.687)',
     'pow(re, 0.678)'),
    ('ergun inertial',
     '1.75 * (1.0 - eps_g) * rho_g * slip / d',
     '1.57 * (1.0 - eps_g) * rho_g * slip / d'),
    ('beta omega dropped',
     'cd0_slip / d * omega;',
     'cd0_slip / d;'),
    ('beta switch',
     'if (eps_g > 0.74) {\n        double omega',
     'if (eps_g > 0.8) {\n        double omega'),
    # deposition, partner choice and wall rules of the hard spheres, soft walls
    ('vs mean',
     'sum[a] / (double)n : 0.0',
     'sum[a] / (double)(n + 1) : 0.0'),
    ('tie to later candidate',
     'if (d2 < bestd2[p] || (d2 == bestd2[p]',
     'if (d2 <= bestd2[p] || (d2 == bestd2[p]'),
    ('partner tie to larger id',
     '(d2 == bestd2[p] && b->id[j] < b->id[bestp[p]])',
     '(d2 == bestd2[p] && b->id[j] > b->id[bestp[p]])'),
    ('walls for paired too',
     'if (paired[p] || !b->wall_hit[p]) continue;',
     'if (!b->wall_hit[p]) continue;'),
    ('lower wall without approach',
     'if (pa < r && va < 0.0) b->wall_hit[p] |= 1 << (2 * a);',
     'if (pa < r) b->wall_hit[p] |= 1 << (2 * a);'),
    ('upper wall approach sign',
     '(double)b->n[a] - pa < r && va > 0.0)',
     '(double)b->n[a] - pa < r && va < 0.0)'),
    ('soft wall lever is r',
     'for (int c = 0; c < 3; ++c) vc[c] = (c < dim ? vp[c] : 0.0) - l * wxn[c];\n                contact_add(b, nrm, l, f, vc, F, T);',
     'for (int c = 0; c < 3; ++c) vc[c] = (c < dim ? vp[c] : 0.0) - r * wxn[c];\n                contact_add(b, nrm, r, f, vc, F, T);'),
    ('pair order descending',
     'if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;',
     'if (a[0] != b[0]) return a[0] < b[0] ? 1 : -1;'),
    # soft-sphere walls, the open outlet, bubble regions
    ('wall damping with m/2',
     'k->eta_w = 2.0 * z * sqrt(k->mp * k->kn);',
     'k->eta_w = 2.0 * z * sqrt(0.5 * k->mp * k->kn);'),
    ('soft outlet closed',
     'if (side == 1 && b->recirculate && a == dim - 1) continue;',
     'if (side == 1 && b->recirculate && a == dim - 1 && 0) continue;'),
    ('freeboard counted',
     'if (top) continue;',
     'if (top && 0) continue;'),
    ('open faces at local density',
     'b->fnew[(size_t)i * nc + x] = feq(b, i, 1.0, uin);',
     'b->fnew[(size_t)i * nc + x] = feq(b, i, b->rho[x], uin);'),
    ('guo second order',
     '+ 9.0 * cu * b->c[i][a]) * b->k.fb[a];',
     '+ 3.0 * cu * b->c[i][a]) * b->k.fb[a];'),
    ('in-cell order by id reversed',
     'if (a->id != b->id) return a->id < b->id ? -1 : 1;',
     'if (a->id != b->id) return a->id < b->id ? 1 : -1;'),
    ('bed voidage from the deposition',
     'se += voidage_of_count(b, b->cell_start[x + 1] - b->cell_start[x], &es, &e2);',
     'se += voidage_of_count(b, b->ntot[x], &es, &e2);'),
    ('set_inlet unscaled',
     'b->inlet_u[j * 3 + a] = inlet_si[j * b->dim + a] * b->uscale;',
     'b->inlet_u[j * 3 + a] = inlet_si[j * b->dim + a];'),
]


def run_one(idx, name, old, new, tmp):
    text = open(SRC).read()
    if text.count(old) != 1:
        return name, None, f"the original text occurs {text.count(old)} times"
    src = os.path.join(tmp, f"mutant{idx}.c")
    lib = os.path.join(tmp, f"mutant{idx}.so")
    with open(src, "w") as fh:
        fh.write(text.replace(old, new, 1))
    oracle_build.build_to(src, lib, quiet=True)
    env = dict(os.environ, LBDPS_ORACLE_LIB=lib)
    # (the pin file's own sampled run of this check is left out, so that a
    # surviving mutant cannot start the check again)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider", "-k", "not mutation_check"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    note = failed[0][7:] if failed else f"pytest exited with status {r.returncode}"
    return name, r.returncode != 0, note


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", "--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("-k", action="append", default=[],
                    help="only mutants whose name contains this (repeatable)")
    args = ap.parse_args()
    todo = [(i, *m) for i, m in enumerate(MUTANTS)
            if not args.k or any(k in m[0] for k in args.k)]
    scratch = os.path.join(ROOT, "_build")     # git-ignored, inside the repository
    os.makedirs(scratch, exist_ok=True)
    with tempfile.TemporaryDirectory(dir=scratch) as tmp:
        with ThreadPoolExecutor(max_workers=max(1, args.jobs)) as pool:
            results = list(pool.map(lambda t: run_one(*t, tmp), todo))
    missed = 0
    for name, caught, note in results:
        mark = "caught" if caught else ("ERROR " if caught is None else "MISSED")
        missed += caught is not True
        print(f"{mark}  {name:26s} {note[:90]}")
    print(f"{len(results) - missed} of {len(results)} caught")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
