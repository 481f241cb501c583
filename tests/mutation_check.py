#!/usr/bin/env python3
"""Mutation check of the oracle's pins (test infrastructure, run by hand).

Plants one plausible mistake at a time in a scratch copy of ``oracle/`` (with ``tests/``,
``synth/`` and ``pytest.ini``), runs the oracle pins (``tests/test_oracle_*.py``) there, and
reports every mistake that no pin catches.  A mistake counts as caught only when a pin fails;
an error (a copy that does not build or collect) is reported on its own.  The mistakes cover
the fit (EM loop, M-step, leave-one-out, posterior, mixture updates), the DQ algebra and the
field, the warp and blend, the node layer (Eqs. 5-15, ARAP, node insertion, the Eq. 8
uncertainty) and the warm-start network.  Two are known not to change any result and are
listed in EXPECTED_SURVIVORS.

    python tests/mutation_check.py [--scratch DIR] [--only GROUP] [--list]

The scratch directory (default: a new temporary directory) is deleted and re-created for every
mistake; the sources in this repository are never modified.
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

EXPECTED_SURVIVORS = {
    'tapclamp': 'an unclamped last bilinear tap has weight 0 wherever it is used',
    'clamp_hi': 'the running average of values up to 255 never exceeds 255',
}

# (group, name, file, text in the file, replacement): one planted mistake each
MUTATIONS = [
    ('core', 'loo', 'oracle/emdq_oracle.c',
     'if (i == j) continue;                    /* leave one out */',
     ''),
    ('core', 'pi_not_pj', 'oracle/emdq_oracle.c',
     'double om = p[j] * exp(-alpha * (dx * dx + dy * dy));\n            W += om;',
     'double om = p[i] * exp(-alpha * (dx * dx + dy * dy));\n            W += om;'),
    ('core', 'sigma2x2', 'oracle/emdq_oracle.c',
     'num / (2.0 * den)',
     'num / den'),
    ('core', 'no2pi', 'oracle/emdq_oracle.c',
     'exp(-e[j] / (2.0 * s2)) / (two_pi * s2)',
     'exp(-e[j] / (2.0 * s2)) / (s2)'),
    ('core', 'dqorder', 'oracle/emdq_oracle.c',
     'qmul(tq, r, d);',
     'qmul(r, tq, d);'),
    ('core', 'scaleinv', 'oracle/emdq_oracle.c',
     'sqrt(vy / vx)',
     'sqrt(vx / vy)'),
    ('core', 'trans', 'oracle/emdq_oracle.c',
     'yb[0] / sc - (cr',
     'yb[0] * sc - (cr'),
    ('core', 'atan_sign', 'oracle/emdq_oracle.c',
     'atan2(S[1][0] - S[0][1]',
     'atan2(S[0][1] - S[1][0]'),
    ('core', 'S_transp', 'oracle/emdq_oracle.c',
     'S[0][1] += om * b0 * a1;',
     'S[0][1] += om * b1 * a0;'),
    ('core', 'fxfy', 'oracle/emdq_oracle.c',
     'double v = (1 - fx) * (1 - fy) * i00 + fx * (1 - fy) * i10 +',
     'double v = (1 - fy) * (1 - fx) * i00 + fy * (1 - fx) * i10 +'),
    ('core', 'cap31', 'oracle/emdq_oracle.c',
     'w + 1.0 < 30.0 ? w + 1.0 : 30.0',
     'w + 1.0 < 31.0 ? w + 1.0 : 31.0'),
    ('core', 'noround', 'oracle/emdq_oracle.c',
     'double r = floor(z + 0.5);',
     'double r = floor(z);'),
    ('core', 'gamma_init', 'oracle/emdq_oracle.c',
     'double g = 0.5;',
     'double g = 0.8;'),
    ('core', 'nonorm', 'oracle/emdq_oracle.c',
     'double n = sqrt(q[0] * q[0] + q[1] * q[1]);',
     'double n = 1.0;'),
    ('core', 'tx_sign', 'oracle/emdq_oracle.c',
     'q[3] = 0.5 * d[2];',
     'q[3] = -0.5 * d[2];'),
    ('core', 'alpha', 'oracle/emdq_oracle.c',
     'return 2e-4 / (s * s);',
     'return 2e-4 / s;'),
    ('core', 'gam_upd', 'oracle/emdq_oracle.c',
     'g = clampd(m / n, 0.05, 0.95);\n        if (dp_trace)',
     'g = 0.5;\n        if (dp_trace)'),
    ('core', 'wcentroid', 'oracle/emdq_oracle.c',
     'xb[0] += om * src[2 * j];',
     'xb[0] += om * dst[2 * j];'),
    ('core', 'c_thresh', 'oracle/emdq_oracle.c',
     'c[j] = p[j] >= 0.5 ? p[j] : 0.0;',
     'c[j] = p[j];'),
    ('core', 'tapclamp', 'oracle/emdq_oracle.c',
     'int x1 = x0 + 1 < fw ? x0 + 1 : fw - 1;',
     'int x1 = x0 + 1;'),
    ('core', 'area_sqrt', 'oracle/emdq_oracle.c',
     '(1.0 - g) / area);',
     '(1.0 - g) / sqrt(area));'),
    ('core', 'no_floor', 'oracle/emdq_oracle.c',
     'return s2 > floor_ ? s2 : floor_;',
     'return s2;'),
    ('core', 'g_no2', 'oracle/emdq_oracle.c',
     'double G = isfinite(e[j]) ? exp(-e[j] / (2.0 * s2))',
     'double G = isfinite(e[j]) ? exp(-e[j] / s2)'),
    ('core', 'p_stuck', 'oracle/emdq_oracle.c',
     'memcpy(p, pn, sizeof(double) * n);',
     ''),
    ('core', 'p0_gamma', 'oracle/emdq_oracle.c',
     'g = clampd(m / n, 0.05, 0.95);\n    } else {',
     'g = 0.5;\n    } else {'),
    ('core', 'e_step_c', 'oracle/emdq_oracle.c',
     'orc_residuals(src, dst, p, q8, n, alpha, e);\n        s2 = sigma2_update',
     'orc_residuals(src, dst, c, q8, n, alpha, e);\n        s2 = sigma2_update'),
    ('nodes', 'beta_s', 'oracle/emdq_oracle.c',
     'return 3e-3 / (s * s);',
     'return 3e-3 / s;'),
    ('nodes', 'unc_sign', 'oracle/emdq_oracle.c',
     'double u = exp(beta * (dx * dx + dy * dy));',
     'double u = exp(-beta * (dx * dx + dy * dy));'),
    ('nodes', 'unc_outliers', 'oracle/emdq_oracle.c',
     'if (!(c[j] > 0.0)) continue;\n        double dx = src[2 * j] - px',
     'double dx = src[2 * j] - px'),
    ('nodes', 'unc_max', 'oracle/emdq_oracle.c',
     'if (u < best) best = u;',
     'if (u > best || best == INFINITY) best = u;'),
    ('nodes', 'cmp_rot', 'oracle/emdq_oracle.c',
     'tho + dth, c * txo',
     'tho - dth, c * txo'),
    ('nodes', 'cmp_tdiv', 'oracle/emdq_oracle.c',
     'dtx / so, sn * txo',
     'dtx * so, sn * txo'),
    ('nodes', 'cmp_rsign', 'oracle/emdq_oracle.c',
     'c * txo - sn * tyo',
     'c * txo + sn * tyo'),
    ('nodes', 'cmp_scale', 'oracle/emdq_oracle.c',
     'row_from_srt(ds * so,',
     'row_from_srt(ds,'),
    ('nodes', 'trk_ds', 'oracle/emdq_oracle.c',
     's2_new[i] = dw[4] * dw[4] * s2_old[i] + du;',
     's2_new[i] = dw[4] * s2_old[i] + du;'),
    ('nodes', 'trk_unc_x0', 'oracle/emdq_oracle.c',
     'const double du = uncertainty_at(c, src, n, p[0], p[1], beta);',
     'const double du = uncertainty_at(c, src, n, x0[2 * i], x0[2 * i + 1], beta);'),
    ('nodes', 'trk_dw_x0', 'oracle/emdq_oracle.c',
     'if (!warp_at(q8, c, src, n, p[0], p[1], alpha, dw)) {',
     'if (!warp_at(q8, c, src, n, x0[2 * i], x0[2 * i + 1], alpha, dw)) {'),
    ('nodes', 'trk_noprop', 'oracle/emdq_oracle.c',
     's2_new[i] = dw[4] * dw[4] * s2_old[i] + du;',
     's2_new[i] = s2_old[i] + du;'),
    ('nodes', 'mrg_eta_sign', 'oracle/emdq_oracle.c',
     'const double eta = exp(-gamma * (dx * dx + dy * dy));',
     'const double eta = exp(gamma * (dx * dx + dy * dy));'),
    ('nodes', 'mrg_sum', 'oracle/emdq_oracle.c',
     'const double sm = 1.0 / (i00 + 2.0 * i01 + i11);',
     'const double sm = 1.0 / (i00 + i01 + i11);'),
    ('nodes', 'mrg_w0', 'oracle/emdq_oracle.c',
     'const double w0 = sm * (i00 + i01)',
     'const double w0 = sm * (i00 - i01)'),
    ('nodes', 'mrg_fallback', 'oracle/emdq_oracle.c',
     'const double *pick = vt <= vl ? wt : wl;',
     'const double *pick = vt <= vl ? wl : wt;'),
    ('nodes', 'mrg_eta_x0', 'oracle/emdq_oracle.c',
     'const double dx = xt[0] - xk[0], dy = xt[1] - xk[1];',
     'const double dx = xt[0] - x0[2 * i], dy = xt[1] - x0[2 * i + 1];'),
    ('nodes', 'mrg_det', 'oracle/emdq_oracle.c',
     'det = vt * vl - a01 * a01;',
     'det = vt * vl + a01 * a01;'),
    ('nodes', 'arap_lam', 'oracle/emdq_oracle.c',
     'const double lam = (1.0 + s2[i]) / (1.0 + 100.0);',
     'const double lam = (1.0 + s2[i]) / 100.0;'),
    ('nodes', 'arap_swap', 'oracle/emdq_oracle.c',
     'average_rows(w_merge + 8 * (size_t)i, 1.0, wa + 8 * (size_t)i, lam, wk + 8 * (size_t)i);',
     'average_rows(w_merge + 8 * (size_t)i, lam, wa + 8 * (size_t)i, 1.0, wk + 8 * (size_t)i);'),
    ('nodes', 'arap_nostop', 'oracle/emdq_oracle.c',
     'if (cost > prev) break;',
     ''),
    ('nodes', 'arap_pos_merge', 'oracle/emdq_oracle.c',
     'for (int i = 0; i < nn; ++i) apply_row(w_out + 8 * (size_t)i,',
     'for (int i = 0; i < nn; ++i) apply_row(w_merge + 8 * (size_t)i,'),
    ('nodes', 'arap_centroid', 'oracle/emdq_oracle.c',
     'orc_arap_fit(x0, xt, nn, alpha, sc, th, t, wa);',
     '{ double *one = malloc(sizeof(double) * (size_t)nn); for (int i = 0; i < nn; ++i) one[i] = 1.0;'
     ' orc_mstep(x0, xt, one, nn, alpha, sc, th, t, wa); free(one); }'),
    ('nodes', 'arap_w_once', 'oracle/emdq_oracle.c',
     'double c0[2] = {w * ex, w * ey};',
     'double c0[2] = {ex, ey};'),
    ('nodes', 'arap_ct_x0', 'oracle/emdq_oracle.c',
     'w * (xt[2 * j] - xt[2 * i]), w * (xt[2 * j + 1] - xt[2 * i + 1])',
     'w * (xt[2 * j] - x0[2 * i]), w * (xt[2 * j + 1] - x0[2 * i + 1])'),
    ('nodes', 'arap_s_inv', 'oracle/emdq_oracle.c',
     'double sc = sqrt(nt) / sqrt(n0);',
     'double sc = sqrt(n0) / sqrt(nt);'),
    ('nodes', 'arap_angle', 'oracle/emdq_oracle.c',
     'double ang = atan2(M[1][0] - M[0][1], M[0][0] + M[1][1]);',
     'double ang = atan2(M[0][1] - M[1][0], M[0][0] + M[1][1]);'),
    ('nodes', 'arap_M_transp', 'oracle/emdq_oracle.c',
     'for (int k = 0; k < 2; ++k) M[r][k] += ct[r] * c0[k];',
     'for (int k = 0; k < 2; ++k) M[r][k] += c0[r] * ct[k];'),
    ('nodes', 'arap_t_w2', 'oracle/emdq_oracle.c',
     '            W += w;\n            tx += w * (xt[2 * j] / sc',
     '            w *= w;\n            W += w;\n            tx += w * (xt[2 * j] / sc'),
    ('nodes', 'arap_t_nos', 'oracle/emdq_oracle.c',
     'ty += w * (xt[2 * j + 1] / sc - (sr',
     'ty += w * (xt[2 * j + 1] - (sr'),
    ('nodes', 'arap_cost_lam', 'oracle/emdq_oracle.c',
     'lam * ((pa[0] - pk[0])',
     '((pa[0] - pk[0])'),
    ('nodes', 'rst_mul', 'oracle/emdq_oracle.c',
     'double b = s2f[j] + exp(beta * (dx * dx + dy * dy));',
     'double b = s2f[j] * exp(beta * (dx * dx + dy * dy));'),
    ('nodes', 'rst_nostart', 'oracle/emdq_oracle.c',
     'double best = s2[i];\n        for (int j = 0; j < m; ++j) {',
     'double best = INFINITY;\n        for (int j = 0; j < m; ++j) {'),
    ('nodes', 'kf_nomean', 'oracle/emdq_oracle.c',
     'out[k] = sum / nn;',
     'out[k] = sum;'),
    ('nodes', 'kf_sq', 'oracle/emdq_oracle.c',
     'sum += hypot(xt[2 * i] - p[0], xt[2 * i + 1] - p[1]);',
     'sum += (xt[2 * i] - p[0]) * (xt[2 * i] - p[0]) + (xt[2 * i + 1] - p[1]) * (xt[2 * i + 1] - p[1]);'),
    ('nodes', 'fu_noprev', 'oracle/emdq_oracle.c',
     's2_out[j] = s2_prev[j] + e[j];',
     's2_out[j] = e[j];'),
    ('nodes', 'fu_ds', 'oracle/emdq_oracle.c',
     's2_out[j] = row[4] * row[4] * s2_prev[j] +',
     's2_out[j] = row[4] * s2_prev[j] +'),
    ('nodes', 'fu_noloo', 'oracle/emdq_oracle.c',
     'orc_residuals(src, dst, c, q8, n, alpha, e);',
     'orc_residuals(src, dst, c, q8, n, 0.0, e);'),
    ('nodes', 'ni_alpha', 'oracle/emdq_oracle.c',
     'if (!warp_at(w, ones, x0, n, pts[2 * k], pts[2 * k + 1], alpha, w_out',
     'if (!warp_at(w, ones, x0, n, pts[2 * k], pts[2 * k + 1], 2.0 * alpha, w_out'),
    ('nodes', 'gamma_s', 'oracle/emdq_oracle.c',
     'return 5e-3 / (s * s);',
     'return 5e-3 / s;'),
    ('nodes', 'hex_dy', 'oracle/__init__.py',
     'dy = spacing * np.sqrt(3.0) / 2.0',
     'dy = spacing / 2.0'),
    ('nodes', 'hex_off', 'oracle/__init__.py',
     'off = 0.5 * spacing if r % 2 else 0.0',
     'off = 0.0'),
    ('nodes', 'hex_radius', 'oracle/__init__.py',
     'm = spacing / np.sqrt(3.0)',
     'm = spacing / 4.0'),
    ('nodes', 'hex_centre', 'oracle/__init__.py',
     'cx, cy = (w - 1) / 2.0, (h - 1) / 2.0',
     'cx, cy = 0.0, 0.0'),
    ('warmstart', 'knn_self', 'oracle/warmstart.py',
     '        d[j] = np.inf\n',
     ''),
    ('warmstart', 'knn_ties', 'oracle/warmstart.py',
     'order = np.lexsort((np.arange(n), d))',
     'order = np.lexsort((-np.arange(n), d))'),
    ('warmstart', 'f1_sign', 'oracle/warmstart.py',
     'np.hypot(*(disp[k] - disp[j]))',
     'np.hypot(*(disp[k] + disp[j]))'),
    ('warmstart', 'f1_desc', 'oracle/warmstart.py',
     'f[j, :K_NN] = np.sort(f1)',
     'f[j, :K_NN] = np.sort(f1)[::-1]'),
    ('warmstart', 'f2_dst', 'oracle/warmstart.py',
     'np.log1p(np.hypot(*(src[k] - src[j])))',
     'np.log1p(np.hypot(*(dst[k] - dst[j])))'),
    ('warmstart', 'f2_nolog', 'oracle/warmstart.py',
     'f2 = [np.log1p(np.hypot(*(src[k] - src[j])))',
     'f2 = [(np.hypot(*(src[k] - src[j])))'),
    ('warmstart', 'relu2', 'oracle/warmstart.py',
     'h2 = np.maximum(a2, 0.0)',
     'h2 = a2'),
    ('warmstart', 'sigmoid', 'oracle/warmstart.py',
     'p = 1.0 / (1.0 + np.exp(-z))',
     'p = 1.0 / (1.0 + np.exp(z))'),
    ('warmstart', 'loss_sign', 'oracle/warmstart.py',
     'np.logaddexp(0.0, z) - y * z',
     'np.logaddexp(0.0, z) + y * z'),
    ('warmstart', 'grad_mean', 'oracle/warmstart.py',
     'dz = (p - y) / B',
     'dz = (p - y)'),
    ('warmstart', 'grad_mask', 'oracle/warmstart.py',
     'dh1 = (dh2 @ W2) * (a1 > 0)',
     'dh1 = (dh2 @ W2)'),
    ('warmstart', 'adam_bias', 'oracle/warmstart.py',
     'mh = m / (1.0 - b1 ** t)',
     'mh = m'),
    ('warmstart', 'adam_v', 'oracle/warmstart.py',
     'v = b2 * v + (1.0 - b2) * g * g',
     'v = b2 * v + (1.0 - b2) * np.abs(g)'),
    ('warp', 'cover_w', 'oracle/emdq_oracle.c',
     'u0 <= fw - 1.0 && u1',
     'u0 <= fw && u1'),
    ('warp', 'cover_neg', 'oracle/emdq_oracle.c',
     'if (!(u0 >= 0.0 && u0',
     'if (!(u0 >= -0.5 && u0'),
    ('warp', 'ytap', 'oracle/emdq_oracle.c',
     'int y1 = y0 + 1 < fh ? y0 + 1 : fh - 1;',
     'int y1 = y0;'),
    ('warp', 'pitch', 'oracle/emdq_oracle.c',
     'frame[(size_t)y0 * frame_pitch + (size_t)x0 * channels + k];',
     'frame[(size_t)y0 * fw * channels + (size_t)x0 * channels + k];'),
    ('warp', 'chan', 'oracle/emdq_oracle.c',
     'double i11 = frame[(size_t)y1 * frame_pitch + (size_t)x1 * channels + k];',
     'double i11 = frame[(size_t)y1 * frame_pitch + (size_t)x1 * channels];'),
    ('warp', 'origin', 'oracle/emdq_oracle.c',
     'canvas + (size_t)(py + oy) * canvas_pitch + 4 * (size_t)(px + ox);',
     'canvas + (size_t)(py + oy) * canvas_pitch + 4 * (size_t)(px - ox);'),
    ('warp', 'wupd', 'oracle/emdq_oracle.c',
     'cp[3] = (uint8_t)(w + 1.0 < 30.0 ? w + 1.0 : 30.0);',
     'cp[3] = (uint8_t)(w < 30.0 ? w : 30.0);'),
    ('warp', 'avg_w', 'oracle/emdq_oracle.c',
     '(w * cp[k] + v) / (w + 1.0)',
     '(w * cp[k] + v) / (w + 2.0)'),
    ('warp', 'ref_w', 'oracle/emdq_oracle.c',
     '            cp[3] = 1;\n        }',
     '            cp[3] = 0;\n        }'),
    ('warp', 'ref_xy', 'oracle/emdq_oracle.c',
     'cp[k] = frame[(size_t)y * frame_pitch + (size_t)x * channels + k];',
     'cp[k] = frame[(size_t)x * frame_pitch + (size_t)y * channels + k];'),
    ('warp', 'fp64_u', 'oracle/emdq_oracle.c',
     'volatile float ux = (float)px + d[0];',
     'volatile double ux = (double)px + (double)d[0];'),
    ('warp', 'clamp_hi', 'oracle/emdq_oracle.c',
     'return r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);',
     'return r < 0.0 ? 0.0 : r;'),
    ('field', 'fld_noc', 'oracle/emdq_oracle.c',
     '        double w = c[i] * exp(-alpha * (dx * dx + dy * dy));\n        sw += w;\n        ss += w * q8[8 * i + 4];',
     '        double w = exp(-alpha * (dx * dx + dy * dy));\n        sw += w;\n        ss += w * q8[8 * i + 4];'),
    ('field', 'fld_sdiv', 'oracle/emdq_oracle.c',
     'orc_apply_warp(ss / sw, q, px, py, xp);',
     'orc_apply_warp(ss, q, px, py, xp);'),
    ('field', 'fld_sq_unw', 'oracle/emdq_oracle.c',
     '        for (int k = 0; k < 4; ++k) sq[k] += w * q8[8 * i + k];\n    }\n    if (!(sw > 0.0) || !isfinite(sw)) {\n        out[0]',
     '        for (int k = 0; k < 4; ++k) sq[k] += q8[8 * i + k];\n    }\n    if (!(sw > 0.0) || !isfinite(sw)) {\n        out[0]'),
    ('field', 'fld_pos', 'oracle/emdq_oracle.c',
     '    out[0] = xp[0] - px;',
     '    out[0] = xp[0];'),
    ('field', 'rot_sign', 'oracle/emdq_oracle.c',
     '    out[0] = s * (c * px - sn * py + tx);',
     '    out[0] = s * (c * px + sn * py + tx);'),
    ('field', 'half_angle', 'oracle/emdq_oracle.c',
     '    *th = 2.0 * atan2(r[3], r[0]);',
     '    *th = atan2(r[3], r[0]);'),
    ('field', 'fld_wx', 'oracle/emdq_oracle.c',
     '        double dx = src[2 * i] - px, dy = src[2 * i + 1] - py;\n        double w = c[i] * exp(-alpha * (dx * dx + dy * dy));\n        sw += w;',
     '        double dx = src[2 * i] - px, dy = src[2 * i + 1] - py;\n        double w = c[i] * exp(-alpha * (dx * dx));\n        sw += w;'),
]


def run_one(scratch: str, file: str, old: str, new: str) -> str:
    shutil.rmtree(scratch, ignore_errors=True)
    os.makedirs(scratch)
    for d in ('oracle', 'synth', 'tests'):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(scratch, d),
                        ignore=shutil.ignore_patterns('__pycache__', '*.so', '*.tmp'))
    shutil.copy(os.path.join(ROOT, 'pytest.ini'), scratch)
    path = os.path.join(scratch, file)
    src = open(path).read()
    if old not in src:
        return 'stale'
    open(path, 'w').write(src.replace(old, new, 1))
    tests = sorted(os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, 'tests', 'test_oracle_*.py')))
    r = subprocess.run([sys.executable, '-m', 'pytest', '-q', '-x', '-p', 'no:cacheprovider', *tests],
                       cwd=scratch, capture_output=True, text=True, timeout=900)
    last = (r.stdout.strip().splitlines() or [''])[-1]
    if ' failed' in last:
        return 'caught'
    if ' error' in last or r.returncode not in (0, 1):
        return 'error'
    return 'survived'


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__.split('\n')[0])
    ap.add_argument('--scratch', default=None, help='scratch directory (re-created per mistake)')
    ap.add_argument('--only', default=None, help='one group: core, field, nodes, warmstart or warp')
    ap.add_argument('--list', action='store_true', help='list the mistakes and exit')
    args = ap.parse_args()
    todo = [m for m in MUTATIONS if args.only in (None, m[0])]
    if args.list:
        for g, name, f, _, _ in todo:
            print(f'{g:10s} {name:16s} {f}')
        return 0
    scratch = args.scratch or tempfile.mkdtemp(prefix='oracle_mutation_')
    bad = []
    try:
        for g, name, f, old, new in todo:
            res = run_one(scratch, f, old, new)
            note = ''
            if res != 'caught':
                note = EXPECTED_SURVIVORS.get(name, '')
                if not (res == 'survived' and note):
                    bad.append(name)
            print(f'{g:10s} {name:16s} {res}{"  (" + note + ")" if note else ""}', flush=True)
    finally:
        shutil.rmtree(scratch, ignore_errors=True)
    caught = len(todo) - len(bad) - sum(1 for m in todo if m[1] in EXPECTED_SURVIVORS)
    print(f'{caught} of {len(todo)} caught; unexpected: {bad or "none"}')
    return 1 if bad else 0


if __name__ == '__main__':
    sys.exit(main())
