"""The oracle's pins catch plausible mistakes (no GPU).

Each entry plants one mistake in a copy of the oracle (a constant of the
opacity rule, the projection or the entropy; a sign in the conic, the
Jacobian or the rotation; an order; a threshold test; a term of the
adjoint; a rule of the objective, the scoring, the top-k selection or the
Exploration Map), runs the pins of ``tests/test_oracle_pins.py`` against
that copy in a scratch directory, and expects at least one of them to
fail.  The repository's own oracle is never modified.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (file, what is wrong, original text, planted text)
MUTANTS = [
    # oracle/gs_oracle.c
    ('oracle/gs_oracle.c', 'dilation 0.2',
     '#define DILATION ((real)0.3)',
     '#define DILATION ((real)0.2)'),
    ('oracle/gs_oracle.c', 'sigma 2.9',
     '#define SIGMA_MUL ((real)3)',
     '#define SIGMA_MUL ((real)2.9)'),
    ('oracle/gs_oracle.c', 'eig floor 0',
     '#define EIG_FLOOR ((real)0.1)',
     '#define EIG_FLOOR ((real)0.0)'),
    ('oracle/gs_oracle.c', 'frustum 1.15',
     '#define FRUSTUM_CLAMP ((real)1.3)',
     '#define FRUSTUM_CLAMP ((real)1.15)'),
    ('oracle/gs_oracle.c', 'alpha max 0.999',
     '#define ALPHA_MAX ((real)0.99)',
     '#define ALPHA_MAX ((real)0.999)'),
    ('oracle/gs_oracle.c', 'alpha min 1/256',
     '#define ALPHA_MIN ((real)1 / (real)255)',
     '#define ALPHA_MIN ((real)1 / (real)256)'),
    ('oracle/gs_oracle.c', 'tstop 1e-3',
     '#define T_STOP ((real)0.0001)',
     '#define T_STOP ((real)0.001)'),
    ('oracle/gs_oracle.c', 'stop on T',
     'if (Tn < T_STOP) break;',
     'if (T < T_STOP) break;'),
    ('oracle/gs_oracle.c', 'pixel centre',
     'const real px = (real)x + (real)0.5, py = (real)y + (real)0.5;',
     'const real px = (real)x, py = (real)y + (real)0.5;'),
    ('oracle/gs_oracle.c', 'cb sign',
     '- p->cb * (dx * dy);',
     '+ p->cb * (dx * dy);'),
    ('oracle/gs_oracle.c', 'drop last sem',
     'for (int j = 0; j < sc->k; ++j) sem[',
     'for (int j = 0; j < sc->k - 1; ++j) sem['),
    ('oracle/gs_oracle.c', 'tie gid desc',
     'return (x->gid > y->gid) - (x->gid < y->gid);',
     'return (x->gid < y->gid) - (x->gid > y->gid);'),
    ('oracle/gs_oracle.c', 'depth sort desc',
     'if (x->depth < y->depth) return -1;',
     'if (x->depth < y->depth) return 1;'),
    ('oracle/gs_oracle.c', 'rect -0.5 off',
     'real xlo = R_CEIL((p->u - (real)0.5) - p->radius);',
     'real xlo = R_CEIL((p->u) - p->radius);'),
    ('oracle/gs_oracle.c', 'J02 sign',
     'p->J02 = -(fx * txc) / tz2;',
     'p->J02 = (fx * txc) / tz2;'),
    ('oracle/gs_oracle.c', 'quat R5 sign',
     'R[5] = (real)2 * (yz - wx);',
     'R[5] = (real)2 * (yz + wx);'),
    ('oracle/gs_oracle.c', 'unc weight',
     'if (sc->unc) u += w * sc->unc[g];',
     'if (sc->unc) u += alpha * sc->unc[g];'),
    ('oracle/gs_oracle.c', 'near >=',
     'if (!(p->tz > znear)) return;',
     'if (!(p->tz >= znear + (real)0.05)) return;'),
    ('oracle/gs_oracle.c', 'entropy ln2',
     'h -= q * log(q);',
     'h -= q * log2(q);'),
    ('oracle/gs_oracle.c', 'clip 0.01',
     'ph[c] = v < 0.001 ? 0.001 : (v > 1.0 ? 1.0 : v);',
     'ph[c] = v < 0.01 ? 0.01 : (v > 1.0 ? 1.0 : v);'),
    ('oracle/gs_oracle.c', 'NS count',
     'if ((real)1 - o.T == 0) ns += 1;',
     'if ((real)1 - o.T < (real)1e-2) ns += 1;'),
    ('oracle/gs_oracle.c', 'clamp branch sign',
     'else { dtz += dJ02 * (fx * p->rxc / tz2); }',
     'else { dtz -= dJ02 * (fx * p->rxc / tz2); }'),
    ('oracle/gs_oracle.c', 'clampy branch sign',
     'else { dtz += dJ12 * (fy * p->ryc / tz2); }',
     'else { dtz -= dJ12 * (fy * p->ryc / tz2); }'),
    ('oracle/gs_oracle.c', 'dB factor',
     'real dB = -dcb * inv + dinv * (real)2 * p->B * inv2;',
     'real dB = -dcb * inv + dinv * p->B * inv2;'),
    ('oracle/gs_oracle.c', 'quat norm grad',
     'gq[0] += (dw - w * dot) / p->qn;',
     'gq[0] += dw / p->qn;'),
    ('oracle/gs_oracle.c', 'opacity grad G->a',
     'e[9] += dalpha * c->G;',
     'e[9] += dalpha * c->a;'),
    ('oracle/gs_oracle.c', 'depth grad w->alpha',
     'e[5] += dd * w;',
     'e[5] += dd * c->alpha;'),
    ('oracle/gs_oracle.c', 'cap branch always',
     'if (c->a < ALPHA_MAX) {',
     'if (1) {'),
    ('oracle/gs_oracle.c', 'sem grad w->T',
     'e[10 + j] += dpj * w;',
     'e[10 + j] += dpj * c->T;'),
    ('oracle/gs_oracle.c', 'eval count before the column test',
     '    if (x < p->x0 || x > p->x1) continue;\n    ++ne;',
     '    ++ne;\n    if (x < p->x0 || x > p->x1) continue;'),
    ('oracle/gs_oracle.c', 'sem detach ignored',
     'if (!sem_detach) gi += gsem;',
     'gi += gsem;'),
    ('oracle/gs_oracle.c', 'scale grad',
     'dR[i * 3 + j] = dM[i * 3 + j] * s[j];',
     'dR[i * 3 + j] = dM[i * 3 + j];'),
    # oracle/mapping_loss.py
    ('oracle/mapping_loss.py', 'sil thresh >=',
     'mg = (sil > SIL_MIN).astype(np.float64)',
     'mg = (sil >= SIL_MIN).astype(np.float64)'),
    ('oracle/mapping_loss.py', 'colour weight 1',
     'W_COLOUR = 0.5 ',
     'W_COLOUR = 1.0 '),
    ('oracle/mapping_loss.py', 'lambda swap',
     'LAM_HD, LAM_COS = 0.8, 0.2',
     'LAM_HD, LAM_COS = 0.2, 0.8'),
    ('oracle/mapping_loss.py', 'mask <=',
     'mask = (h < np.log(k)).astype(np.float64)',
     'mask = (h <= np.log(k)).astype(np.float64)'),
    ('oracle/mapping_loss.py', 'mask log k+1',
     'mask = (h < np.log(k)).astype(np.float64)',
     'mask = (h < np.log(k + 1)).astype(np.float64)'),
    ('oracle/mapping_loss.py', 'hd no half',
     'd_hd = np.sqrt(0.5 * ((sq - sp) ** 2).sum(-1))',
     'd_hd = np.sqrt(((sq - sp) ** 2).sum(-1))'),
    ('oracle/mapping_loss.py', 'sem sum not mean',
     'loss = loss_geo + term.sum() / npix',
     'loss = loss_geo + term.sum()'),
    ('oracle/mapping_loss.py', 'dcos sign',
     'grad = mask[..., None] * (LAM_HD * dhd - LAM_COS * dcos)',
     'grad = mask[..., None] * (LAM_HD * dhd + LAM_COS * dcos)'),
    ('oracle/mapping_loss.py', 'dhd sign',
     '(sp - sq) / (2.0 * sp)',
     '(sq - sp) / (2.0 * sp)'),
    ('oracle/mapping_loss.py', 'dhd sqrt factor',
     '(sp - sq) / (2.0 * sp)',
     '(sp - sq) / sp'),
    ('oracle/mapping_loss.py', 'dcos second term sign',
     '- (cos / np.maximum(npn * npn, EPS_DIV))[..., None] * p',
     '+ (cos / np.maximum(npn * npn, EPS_DIV))[..., None] * p'),
    ('oracle/mapping_loss.py', 'dcos norm not squared',
     'np.maximum(npn * npn, EPS_DIV)',
     'np.maximum(npn, EPS_DIV)'),
    ('oracle/mapping_loss.py', 'entropy sign',
     'h = -qlogq.sum(-1)',
     'h = qlogq.sum(-1)'),
    ('oracle/mapping_loss.py', 'depth grad unmasked',
     'd_depth = mg * np.sign(e_d)',
     'd_depth = np.sign(e_d)'),
    ('oracle/mapping_loss.py', 'colour grad weight',
     'd_rgb = W_COLOUR * mg[..., None] * np.sign(e_c)',
     'd_rgb = mg[..., None] * np.sign(e_c)'),
    ('oracle/mapping_loss.py', 'sem grad not mean',
     'd_sem = g / npix',
     'd_sem = g'),
    ('oracle/mapping_loss.py', 'cos norm q twice',
     'den = nq * npn',
     'den = nq * nq'),
    ('oracle/mapping_loss.py', 'negative P as |P|',
     'pc = np.maximum(p, 0.0)',
     'pc = np.abs(p)'),
    ('oracle/mapping_loss.py', 'geometry mean',
     'loss_geo = (mg * (np.abs(e_d) + W_COLOUR * np.abs(e_c).sum(-1))).sum()',
     'loss_geo = (mg * (np.abs(e_d) + W_COLOUR * np.abs(e_c).sum(-1))).mean()'),
    ('oracle/mapping_loss.py', 'colour channel mean',
     'W_COLOUR * np.abs(e_c).sum(-1))).sum()',
     'W_COLOUR * np.abs(e_c).mean(-1))).sum()'),
    # oracle/explore.py
    ('oracle/explore.py', 'prune >',
     'keep = ns >= prune_frac * np.asarray(npix, np.float64)',
     'keep = ns > prune_frac * np.asarray(npix, np.float64)'),
    ('oracle/explore.py', 'prune frac 0.05',
     'PRUNE_FRAC = 0.005',
     'PRUNE_FRAC = 0.05'),
    ('oracle/explore.py', 'mov not 1-',
     'mov = 1.0 - softmax(dist)',
     'mov = softmax(dist)'),
    ('oracle/explore.py', 'igeo no log',
     'igeo = softmax(np.log(ns))',
     'igeo = softmax(ns)'),
    ('oracle/explore.py', 'best ties last',
     'if keep[v] and (best < 0 or iv[v] > iv[best]):',
     'if keep[v] and (best < 0 or iv[v] >= iv[best]):'),
    ('oracle/explore.py', 'fib golden angle',
     'phi = math.pi * (3.0 - math.sqrt(5.0)) * i',
     'phi = math.pi * (3.0 - math.sqrt(4.9)) * i'),
    ('oracle/explore.py', 'fib z offset',
     'z = 1.0 - (2.0 * i + 1.0) / n',
     'z = 1.0 - (2.0 * i) / n'),
    ('oracle/explore.py', 'right axis flip',
     'right = np.cross(d, up)',
     'right = np.cross(up, d)'),
    ('oracle/explore.py', 'lattice floor',
     'pts.add((math.floor(x / step + 0.5), math.floor(y / step + 0.5), hi))',
     'pts.add((math.floor(x / step), math.floor(y / step + 0.5), hi))'),
    ('oracle/explore.py', 'band <',
     'if abs(z - h) <= band:',
     'if abs(z - h) < band:'),
    ('oracle/explore.py', 'semantic factor from U',
     'ns, sh = sums[:, 2], sums[:, 1]',
     'ns, sh = sums[:, 2], sums[:, 0]'),
    ('oracle/explore.py', 'N_S from column 0',
     'ns, sh = sums[:, 2], sums[:, 1]',
     'ns, sh = sums[:, 0], sums[:, 1]'),
    ('oracle/explore.py', 'no N_S: uniform',
     'igeo = np.zeros_like(ns)',
     'igeo = np.full_like(ns, 1.0 / len(ns))'),
    ('oracle/explore.py', 'distance squared',
     'dist = np.linalg.norm(np.asarray(positions, np.float64) - np.asarray(current, np.float64), axis=1)',
     'dist = ((np.asarray(positions, np.float64) - np.asarray(current, np.float64)) ** 2).sum(1)'),
    ('oracle/explore.py', 'best ignores pruning',
     'if keep[v] and (best < 0 or iv[v] > iv[best]):',
     'if (best < 0 or iv[v] > iv[best]):'),
    ('oracle/explore.py', 'down axis flip',
     'down = np.cross(d, right)',
     'down = np.cross(right, d)'),
    ('oracle/explore.py', 'translation sign',
     '(-r @ np.asarray(position, np.float64))',
     '(r @ np.asarray(position, np.float64))'),
    ('oracle/explore.py', 'fib radius',
     'r = np.sqrt(np.maximum(0.0, 1.0 - z * z))',
     'r = np.maximum(0.0, 1.0 - z * z)'),
    ('oracle/explore.py', 'height index as height',
     'out = [(i * step, j * step, hs[hi]) for i, j, hi in sorted(pts)]',
     'out = [(i * step, j * step, float(hi)) for i, j, hi in sorted(pts)]'),
    ('oracle/explore.py', 'score without motion',
     'iv = mov * igeo * isem',
     'iv = igeo * isem'),
    ('oracle/explore.py', 'lattice y floor',
     'pts.add((math.floor(x / step + 0.5), math.floor(y / step + 0.5), hi))',
     'pts.add((math.floor(x / step + 0.5), math.floor(y / step), hi))'),
    # oracle/sparse.py
    ('oracle/sparse.py', 'ties high id',
     'order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, :k]',
     'order = np.lexsort((-np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, :k]'),
    ('oracle/sparse.py', 'nan first',
     'key = np.where(np.isnan(sel), -np.inf, sel)',
     'key = np.where(np.isnan(sel), np.inf, sel)'),
    ('oracle/sparse.py', 'gather invalid',
     'if 0 <= ids[i, l] < m:',
     'if 0 <= ids[i, l] <= m - 1 and ids[i, l] != 0:'),
    ('oracle/sparse.py', 'lowest kept',
     'order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, :k]',
     'order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), key), axis=1)[:, :k]'),
    ('oracle/sparse.py', 'largest skipped',
     'order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, :k]',
     'order = np.lexsort((np.broadcast_to(np.arange(m), key.shape), -key), axis=1)[:, 1:k + 1]'),
    ('oracle/sparse.py', 'init rows ignored',
     'sel = p[r].astype(np.float64)',
     'sel = p[np.arange(len(r))].astype(np.float64)'),
    ('oracle/sparse.py', 'gather rows ignored',
     'out[i, l] = p[r[i], ids[i, l]]',
     'out[i, l] = p[i, ids[i, l]]'),
    # oracle/voxel.py
    ('oracle/voxel.py', 'pixel centre',
     'xc = (u + 0.5 - float(np.float32(cam.cx))) / float(np.float32(cam.fx)) * de',
     'xc = (u - float(np.float32(cam.cx))) / float(np.float32(cam.fx)) * de'),
    ('oracle/voxel.py', 'max depth hit <',
     'hit = d <= float(np.float32(max_depth))',
     'hit = d < float(np.float32(max_depth)) - 0.5'),
    ('oracle/voxel.py', 'occupied loses',
     'return np.where(bits & 2, 2, np.where(bits & 1, 1, 0)).astype(np.uint8)',
     'return np.where(bits & 1, 1, np.where(bits & 2, 2, 0)).astype(np.uint8)'),
    ('oracle/voxel.py', 'new free prev',
     'z, y, x = np.nonzero((cur == 1) & (prev == 0))',
     'z, y, x = np.nonzero((cur == 1) & (prev != 1))'),
    ('oracle/voxel.py', 'zero depth kept',
     'if not (d > 0.0) or not math.isfinite(d):',
     'if not (d >= 0.0) or not math.isfinite(d):'),
    ('oracle/voxel.py', 'camera centre sign',
     'return -r.T @ t, r',
     'return r.T @ t, r'),
    ('oracle/voxel.py', 'rotation not transposed',
     'p = r.T @ np.array([xc, yc, de]) + o',
     'p = r @ np.array([xc, yc, de]) + o'),
    ('oracle/voxel.py', 'pixel centre y',
     'yc = (v + 0.5 - float(np.float32(cam.cy)))',
     'yc = (v - float(np.float32(cam.cy)))'),
    ('oracle/voxel.py', 'ray instead of segment',
     't1 = np.ones(lo.shape[0])',
     't1 = np.full(lo.shape[0], np.inf)'),
    ('oracle/voxel.py', 'end voxel rounded',
     'end = np.floor(b).astype(np.int64)',
     'end = np.round(b).astype(np.int64)'),
    ('oracle/voxel.py', 'slab entry',
     't0 = np.maximum(t0, np.minimum(ta, tb))',
     't0 = np.maximum(t0, np.maximum(ta, tb))'),
    ('oracle/voxel.py', 'new free centre',
     'org[0] + (x + 0.5) * voxel',
     'org[0] + x * voxel'),
]


def _sandbox(dst):
    """A directory holding what the pins import: the oracle, the input
    generator and the pins themselves."""
    os.makedirs(os.path.join(dst, "tests"))
    os.makedirs(os.path.join(dst, "paper_2506_00225_gb300"))
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ("tests/test_oracle_pins.py", "tests/conftest.py", "pytest.ini", "paper_2506_00225_gb300/__init__.py",
              "paper_2506_00225_gb300/scenes.py"):
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))


def _run_pins(d):
    # the pins' scenes are tiny: one OpenMP thread each, several copies at once
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x", "-p",
                        "no:cacheprovider"], cwd=d, capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    return r.returncode, r.stdout[-400:]


def _mutant_survives(base, i):
    f, name, old, new = MUTANTS[i]
    d = os.path.join(base, f"m{i:02d}")
    _sandbox(d)
    path = os.path.join(d, f)
    src = open(path).read()
    assert src.count(old) == 1, (f, name, "the original text is no longer in the oracle")
    open(path, "w").write(src.replace(old, new))
    rc, out = _run_pins(d)
    shutil.rmtree(d, ignore_errors=True)
    return (name, out) if rc == 0 else None


def test_planted_oracle_mistakes_fail_a_pin(tmp_path):
    base = str(tmp_path)
    clean = os.path.join(base, "clean")
    _sandbox(clean)
    rc, out = _run_pins(clean)
    assert rc == 0, "the pins must pass on the unmodified oracle copy:\n" + out
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        survivors = [s for s in ex.map(lambda i: _mutant_survives(base, i), range(len(MUTANTS))) if s]
    assert not survivors, survivors
