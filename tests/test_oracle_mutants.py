"""Mutation check of the oracle's pins: each case plants one plausible
mistake in a copy of the oracle's C source (a dropped term, a wrong sign,
factor or exponent, transposed operands, a wrong index order), builds that
copy on the CPU, and runs the oracle's pin files against it in a subprocess
(``SPH_ORACLE_LIB`` makes ``oracle.lib()`` load the copy).  Every mistake
must make at least one pin fail.  The same is done for the reference
adjoint's PyTorch restatement of the step (``oracle/adjoint.py``): a copy of
the ``oracle`` package with one mistake in it, in a temporary tree, against
``tests/test_adjoint_oracle.py``.  The product code is not involved; the
mistakes exist only in temporary copies.

A case whose original text no longer occurs exactly once in the oracle
fails, so the list follows the source."""
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sph_oracle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_2d.py", "tests/test_oracle_periodic.py",
             "tests/test_oracle_probes.py"]

# (what the mistake is, original text, mistaken text)
MUTANTS = [
    ('kernel normalisation',
     '21.0 / (16.0 * PI * h * h * h)',
     '21.0 / (15.0 * PI * h * h * h)'),
    ('kernel power dropped',
     'return wendland_alpha(h, dim) * t * t * t * t * (2.0 * q + 1.0);',
     'return wendland_alpha(h, dim) * t * t * t * (2.0 * q + 1.0);'),
    ('dW/dr sign',
     'return -5.0 * wendland_alpha',
     'return 5.0 * wendland_alpha'),
    ('Tait exponent',
     '(pow(rho / ph->rho0, gamma_tait) - 1.0)',
     '(pow(rho / ph->rho0, gamma_tait - 1.0) - 1.0)'),
    ('Riemann U* sign',
     'double Ustar = U_bar + 0.5 * (pL - pR) / (c * rho_bar);',
     'double Ustar = U_bar + 0.5 * (pR - pL) / (c * rho_bar);'),
    ('limiter factor',
     'fmin(3.0 * fmax(UL - UR, 0.0), c)',
     'fmin(2.0 * fmax(UL - UR, 0.0), c)'),
    ('P_bar operands',
     'double P_bar = (rhoL * pR + rhoR * pL) / (rhoL + rhoR);',
     'double P_bar = (rhoL * pL + rhoR * pR) / (rhoL + rhoR);'),
    ('wall hydrostatic term dropped',
     'c->num += (s->p[f] + s->rho[f] * gr) * w;',
     'c->num += s->p[f] * w;'),
    ('wall hydrostatic sign',
     'c->num += (s->p[f] + s->rho[f] * gr) * w;',
     'c->num += (s->p[f] - s->rho[f] * gr) * w;'),
    ('multi-phase wall weight',
     'double w = (s->P.n_phases > 1) ? W / s->rho[f] : W;',
     'double w = W;'),
    ('continuity factor 2',
     'c->sum += 2.0 * rho_i * (m_j / rho_j) * dot;',
     'c->sum += rho_i * (m_j / rho_j) * dot;'),
    ('continuity mixture transposed',
     'double vmix = (rho_i * v_i[d] + rho_j * v_j[d]) / (rho_i + rho_j);',
     'double vmix = (rho_j * v_i[d] + rho_i * v_j[d]) / (rho_i + rho_j);'),
    ('momentum rho_j -> rho_i',
     '-2.0 * m_j * pstar / (s->rho[i] * s->rho[j]) * gw[d]',
     '-2.0 * m_j * pstar / (s->rho[i] * s->rho[i]) * gw[d]'),
    ('wall p* operands',
     'double pstar = (rho_i * p_w + rho_w * p_i) / (rho_i + rho_w);',
     'double pstar = (rho_i * p_i + rho_w * p_w) / (rho_i + rho_w);'),
    ('penalty lambda power',
     '(1.0 - delta) * (1.0 - delta) / dx',
     '(1.0 - delta) / dx'),
    ('penalty delta factor',
     'double delta = -2.0 * r / dx * en;',
     'double delta = -1.0 * r / dx * en;'),
    ('penalty delta unsigned',
     'double delta = -2.0 * r / dx * en;',
     'double delta = 2.0 * r / dx * fabs(en);'),
    ('penalty delta sign',
     'double delta = -2.0 * r / dx * en;',
     'double delta = 2.0 * r / dx * en;'),
    ('penalty fluid-facing side',
     'if (rwf[0] * n[0] + rwf[1] * n[1] + rwf[2] * n[2] < 0.0) c->front = 1;',
     'if (rwf[0] * n[0] + rwf[1] * n[1] + rwf[2] * n[2] > 0.0) c->front = 1;'),
    ('penalty fluid-facing ignored',
     'if (phi->penalty && s->wfront[w] && r > 1e-6 * s->P.dp) {',
     'if (phi->penalty && r > 1e-6 * s->P.dp) {'),
    ('viscosity eta',
     '(r * r + 0.01 * s->P.h * s->P.h)',
     '(r * r + 0.1 * s->P.h * s->P.h)'),
    ('viscosity sign',
     'c->a[d] += k * (c->vel[3 * i + d] - v_j[d]);',
     'c->a[d] -= k * (c->vel[3 * i + d] - v_j[d]);'),
    ('reinit free-surface factor',
     'fmax(0.0, rho_star - rho_num) * ph->rho0 / rho_star',
     'fmax(0.0, rho_star - rho_num)'),
    ('first kick full',
     '            s->v[3 * i + d] += 0.5 * dt * s->a[3 * i + d];\n            s->x[3 * i + d] += dt * s->v[3 * i + d];',
     '            s->v[3 * i + d] += dt * s->a[3 * i + d];\n            s->x[3 * i + d] += dt * s->v[3 * i + d];'),
    ('body-force dt limit',
     'dt = fmin(dt, s->P.cfl * sqrt(s->P.h / gn));',
     'dt = fmin(dt, s->P.cfl * sqrt(2.0 * s->P.h / gn));'),
    ('nearest image',
     'r[d] -= L * floor(r[d] / L + 0.5);',
     'r[d] -= L * floor(r[d] / L);'),
    ('cutoff shrunk',
     'if (r2 >= rc2 || r2 == 0.0) continue;',
     'if (r2 >= 0.95 * rc2 || r2 == 0.0) continue;'),
    ('wall normal sign',
     'c->psi[d] -= V * g[d];',
     'c->psi[d] += V * g[d];'),
    ('cell key axes',
     'return (uint32_t)(((int64_t)c[2] * s->nc[1] + c[1]) * s->nc[0] + c[0]);',
     'return (uint32_t)(((int64_t)c[0] * s->nc[1] + c[1]) * s->nc[2] + c[2]);'),
    ('summation self term',
     'sum_ctx c = {s, W_of(s, 0.0)};',
     'sum_ctx c = {s, 0.0};'),
    ('sensor volume',
     'double Vj = ph->rho0 * V0 / s->rho[j];',
     'double Vj = V0;'),
    ('sensor normalisation',
     'if (p_out) p_out[k] = sw > 0.0 ? spw / sw : 0.0;',
     'if (p_out) p_out[k] = spw;'),
    ('excitation sign',
     's->geff[d] = s->P.g[d] + s->ex_amp[d] * w * w * sw;',
     's->geff[d] = s->P.g[d] - s->ex_amp[d] * w * w * sw;'),
    ('periodic wrap',
     'if (u < 0.0) u += L;',
     'if (u < 0.0) u += 0.5 * L;'),
    ('hydrostatic init',
     'double p = P->phase[k].rho0 * gz * (P->phase[k].z_top - z);',
     'double p = P->phase[k].rho0 * gz * (z - P->phase[k].z_top);'),
    ('stacked phases',
     'p += P->phase[m].rho0 * gz * (P->phase[m].z_top - P->phase[m - 1].z_top);',
     'p += P->phase[k].rho0 * gz * (P->phase[m].z_top - P->phase[m - 1].z_top);'),
    ('E_kin factor',
     'ek += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);',
     'ek += m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);'),
    ('E_pot sign',
     'ep -= m * (s->P.g[0] * x[0] + s->P.g[1] * x[1] + s->P.g[2] * x[2]);',
     'ep += m * (s->P.g[0] * x[0] + s->P.g[1] * x[1] + s->P.g[2] * x[2]);'),
    ('gauge interpolation',
     'out = i == K ? r[2] : r[2] + dz * (phi - 0.5) / (phi - phi_above);',
     'out = r[2];'),
    ('wall density floor',
     's->rhow[2 * w + k] = pw < p_half ? 0.5 * ph->rho0',
     's->rhow[2 * w + k] = pw < p_half ? 0.4 * ph->rho0'),
    ('CFL speed term',
     'double dt = s->P.cfl * s->P.h / (s->P.c0 + max_speed(s));',
     'double dt = s->P.cfl * s->P.h / s->P.c0;'),
    ('reinit number density',
     'double rho_num = ph->rho0 * s->sigma[i] / s->sigma0;',
     'double rho_num = ph->rho0 * s->sigma[i] / (s->sigma0 * 1.001);'),
    ('second kick dropped',
     '        for (int d = 0; d < 3; d++) s->v[3 * i + d] += 0.5 * dt * s->a[3 * i + d];\n    s->step++;',
     '        for (int d = 0; d < 3; d++) s->v[3 * i + d] += 0.0 * dt * s->a[3 * i + d];\n    s->step++;'),
    ('Ustar diffusion factor',
     'double Ustar = U_bar + 0.5 * (pL - pR) / (c * rho_bar);',
     'double Ustar = U_bar + (pL - pR) / (c * rho_bar);'),
    ('penalty side',
     'double Ppen = s->P.gamma_p * lambda * fabs(p_i * en);',
     'double Ppen = s->P.gamma_p * lambda * p_i * en;'),
    ('2-D normalisation',
     'return dim == 2 ? 7.0 / (4.0 * PI * h * h) :',
     'return dim == 2 ? 7.0 / (3.0 * PI * h * h) :'),
    ('2-D lattice sum',
     'int KY = dim == 2 ? 0 : K;',
     'int KY = K;'),
    ('gauge phase filter',
     'if (!in_grid(s, j) || s->phase[j] != 0) continue;',
     'if (!in_grid(s, j)) continue;'),
    ('gauge top sample',
     'int64_t K = (int64_t)floor((zhi - zlo) / dz);',
     'int64_t K = (int64_t)floor((zhi - zlo) / dz) - 1;'),
    ('body force at t^n',
     '    s->t += dt;\n    body_force(s, s->t);',
     '    body_force(s, s->t);\n    s->t += dt;'),
    ('reinit phase of the cycle',
     's->step % s->P.reinit_every == 0) reinit_density(s);',
     's->step % s->P.reinit_every == 1) reinit_density(s);'),
    ('periodic cell key wrap dropped',
     '            if (c[d] >= s->nc[d]) c[d] -= s->nc[d];\n',
     ''),
    ('linear EOS c^2',
     'return c0 * c0 * (rho - ph->rho0);',
     'return c0 * (rho - ph->rho0);'),
    ('summation without walls',
     '    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, sum_visit_w, &c);\n',
     ''),
    ('sigma without walls',
     '    for_neighbors(s, s->x + 3 * i, s->xw, s->order_w, s->start_w, sigma_visit_w, &c);\n',
     ''),
    ('stencil x range',
     '            for (int dx = -1; dx <= 1; dx++) {',
     '            for (int dx = -1; dx <= 0; dx++) {'),
    ('periodic stencil wrap',
     'if (is_periodic(s, d)) q[d] = (q[d] + s->nc[d]) % s->nc[d];',
     'if (is_periodic(s, d)) q[d] = q[d] % s->nc[d];'),
    ('self pair kept',
     'if (r2 >= rc2 || r2 == 0.0) continue; /* self and r = 0 skipped */',
     'if (r2 >= rc2) continue; /* self and r = 0 skipped */'),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutants")
    with open(os.path.join(ROOT, "oracle", "sph_oracle.h")) as fh, open(d / "sph_oracle.h", "w") as out:
        out.write(fh.read())
    return d


@pytest.mark.parametrize("name,original,mistaken", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(workdir, name, original, mistaken):
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(original) == 1, f"the text of case {name!r} no longer occurs once in the oracle"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_file = workdir / f"{tag}.c"
    so_file = workdir / f"{tag}.so"
    c_file.write_text(src.replace(original, mistaken))
    subprocess.check_call(oracle.compile_command(str(c_file), str(so_file)))
    run = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider"],
                         cwd=ROOT, env=dict(os.environ, SPH_ORACLE_LIB=str(so_file)),
                         capture_output=True, text=True, timeout=600)
    assert run.returncode == 1, f"no pin caught: {name}\n{run.stdout[-2000:]}"


# (what the mistake is, original text, mistaken text) in oracle/adjoint.py
ADJOINT_MUTANTS = [
    ('kernel normalisation',
     'return 21.0 / (16.0 * math.pi * h ** 3) * t ** 4 * (2.0 * q + 1.0)',
     'return 21.0 / (15.0 * math.pi * h ** 3) * t ** 4 * (2.0 * q + 1.0)'),
    ('dW/dr sign',
     'return -5.0 * 21.0 / (16.0 * math.pi * h ** 3) * q * t ** 3 / h',
     'return 5.0 * 21.0 / (16.0 * math.pi * h ** 3) * q * t ** 3 / h'),
    ('Tait exponent',
     '((rho / P.rho0) ** P.gamma_tait - 1.0)',
     '((rho / P.rho0) ** (P.gamma_tait - 1.0) - 1.0)'),
    ('Riemann U* sign',
     'Ustar = U_bar + 0.5 * (pL - pR) / (c * rho_bar)',
     'Ustar = U_bar + 0.5 * (pR - pL) / (c * rho_bar)'),
    ('limiter factor',
     'beta = torch.minimum(3.0 * torch.clamp(UL - UR, min=0.0), c * torch.ones_like(UL))',
     'beta = torch.minimum(2.0 * torch.clamp(UL - UR, min=0.0), c * torch.ones_like(UL))'),
    ('P_bar operands',
     'P_bar = (rhoL * pR + rhoR * pL) / rs',
     'P_bar = (rhoL * pL + rhoR * pR) / rs'),
    ('mixture transposed',
     'vmix = (rho[i][:, None] * v_i + rho_j[:, None] * v_j) / (rho[i] + rho_j)[:, None]',
     'vmix = (rho_j[:, None] * v_i + rho[i][:, None] * v_j) / (rho[i] + rho_j)[:, None]'),
    ('continuity factor 2',
     'out.index_add_(0, i, 2.0 * rho[i] * (m / rho_j) * dot)',
     'out.index_add_(0, i, rho[i] * (m / rho_j) * dot)'),
    ('wall hydrostatic sign',
     '(p[wi] + rho[wi] * (rwf @ P.g)) * Wk',
     '(p[wi] - rho[wi] * (rwf @ P.g)) * Wk'),
    ('wall density floor',
     'p_half = eos_p(0.5 * P.rho0 * torch.ones_like(pw), P, c0)',
     'p_half = eos_p(0.4 * P.rho0 * torch.ones_like(pw), P, c0)'),
    ('momentum rho_j -> rho_i',
     'a = a.index_add(0, fi, (-2.0 * m * pstar / (rho[fi] * rho[fj]))[:, None] * gw)',
     'a = a.index_add(0, fi, (-2.0 * m * pstar / (rho[fi] * rho[fi]))[:, None] * gw)'),
    ('wall p* operands',
     'pstar = (rho_i * p_w + rho_w * p_i) / (rho_i + rho_w)',
     'pstar = (rho_i * p_i + rho_w * p_w) / (rho_i + rho_w)'),
    ('viscosity sign',
     'a = a.index_add(0, fi, kv[:, None] * (v[fi] - v[fj]))',
     'a = a.index_add(0, fi, kv[:, None] * (v[fj] - v[fi]))'),
    ('wall viscosity dropped',
     'a = a.index_add(0, wi, kv[:, None] * v[wi])',
     'a = a.index_add(0, wi, 0.0 * kv[:, None] * v[wi])'),
    ('penalty lambda power',
     'lam = torch.where(act, (1.0 - delta) ** 2 / dx, torch.zeros_like(delta))',
     'lam = torch.where(act, (1.0 - delta) / dx, torch.zeros_like(delta))'),
    ('penalty delta factor',
     'delta = 2.0 * rn / dx',
     'delta = rn / dx'),
    ('penalty delta unsigned',
     'delta = 2.0 * rn / dx',
     'delta = 2.0 * torch.abs(rn) / dx'),
    ('penalty fluid-facing ignored',
     'act = facing[ww] & (delta < 1.0) & (r > 1e-6 * dx)',
     'act = (delta < 1.0) & (r > 1e-6 * dx)'),
    ('reinit factor',
     'return rho_num + torch.clamp(rho - rho_num, min=0.0) * P.rho0 / rho',
     'return rho_num + torch.clamp(rho - rho_num, min=0.0)'),
    ('first kick full',
     'vh = S["v"] + 0.5 * dt * S["a"]',
     'vh = S["v"] + dt * S["a"]'),
    ('second kick full',
     'v1 = vh + 0.5 * dt * a',
     'v1 = vh + dt * a'),
    ('continuity at old densities',
     'a = momentum(x, vh, rho1, p1, pw, rhow, P, c0, gamma_p, mu, pairs)',
     'a = momentum(x, vh, rho, p, pw, rhow, P, c0, gamma_p, mu, pairs)'),
    ('nearest image',
     'k = torch.where(P.period > 0, torch.round(r.detach() / L), torch.zeros_like(r))',
     'k = torch.where(P.period > 0, torch.floor(r.detach() / L), torch.zeros_like(r))'),
    ('number density self term',
     's = torch.full((n,), float(W(torch.tensor(0.0, dtype=F64), P.h)), dtype=F64)',
     's = torch.zeros((n,), dtype=F64)'),
    ('reinit cycle',
     'P.reinit_every > 0 and n % P.reinit_every == 0)',
     'P.reinit_every > 0 and n % P.reinit_every == 1)'),
    ('no wrap after drift',
     'x = wrap(S["x"] + dt * vh, P)',
     'x = S["x"] + dt * vh'),
    ('wall pressure at old density',
     'pw, rhow = wall_pressure(x, rho1, p1, P, c0, pairs[1], nw)',
     'pw, rhow = wall_pressure(x, rho, p, P, c0, pairs[1], nw)'),
    ('sigma at old positions',
     'sigma = number_density(x, P, pairs, x.shape[0])\n    return {"x": x, "v": v1',
     'sigma = number_density(S["x"], P, pairs, x.shape[0])\n    return {"x": x, "v": v1'),
    ('continuity with v^n',
     'drdt = continuity(x, vh, rho, p, S["pw"], S["rhow"], P, c0, pairs)',
     'drdt = continuity(x, S["v"], rho, p, S["pw"], S["rhow"], P, c0, pairs)'),
    ('number density without walls',
     '    return s.index_add(0, wi, W(r, P.h))',
     '    return s'),
]


@pytest.mark.parametrize("name,original,mistaken", ADJOINT_MUTANTS, ids=[m[0] for m in ADJOINT_MUTANTS])
def test_a_planted_mistake_in_the_reference_adjoint_fails_a_pin(tmp_path, name, original, mistaken):
    pytest.importorskip("torch")
    pytest.importorskip("scipy")
    with open(os.path.join(ROOT, "oracle", "adjoint.py")) as fh:
        src = fh.read()
    assert src.count(original) == 1, f"the text of case {name!r} no longer occurs once in the adjoint"
    tree = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), tree / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (tree / "oracle" / "adjoint.py").write_text(src.replace(original, mistaken))
    os.symlink(os.path.join(ROOT, "paper_2110_02621_gb300"), tree / "paper_2110_02621_gb300")
    (tree / "tests").mkdir()
    for f in ("conftest.py", "test_adjoint_oracle.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tree / "tests" / f)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tree / "pytest.ini")
    run = subprocess.run([sys.executable, "-m", "pytest", "tests/test_adjoint_oracle.py", "-x", "-q",
                          "-p", "no:cacheprovider"],
                         cwd=tree, env=dict(os.environ, SPH_ORACLE_LIB=oracle.build()),
                         capture_output=True, text=True, timeout=600)
    assert run.returncode == 1, f"no pin caught: {name}\n{run.stdout[-2000:]}"
