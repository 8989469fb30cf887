"""Pins of the circuit generator (the input both sampler and oracle consume).

* Table III of the paper: 1q/2q/M/rows for 10 codes x 2 operations (80 exact
  integers) with 4 rounds before and 3 after; DEM columns (a soft pin that
  depends on the syndrome schedule) exactly for the surface codes.
* Supplementary Table S1 / "Bivariate Bicycle Codes": n, k of every BB code,
  H_X H_Z^T = 0, row weight 6.
* Every detector and observable of every generated circuit is deterministic
  (gauge-randomised noiseless audit).
"""
import numpy as np
import pytest

from conftest import golden_rows
from paper_2504_05611_gb300 import circuits as C

T3 = {r[0]: [int(v) for v in r[1:]] for r in golden_rows("table_iii_counts.txt")}
CODES = {r[0]: tuple(int(v) for v in r[1:]) for r in golden_rows("codes.txt")}


def gf2_rank_plain(m):
    """Independent GF(2) rank (bit-packed Python ints), not the generator's."""
    rows = [int("".join(str(int(b)) for b in row), 2) for row in np.asarray(m) % 2]
    rank = 0
    while rows:
        pivot = max(rows)
        rows.remove(pivot)
        if pivot == 0:
            continue
        rank += 1
        top = pivot.bit_length() - 1
        rows = [r ^ pivot if (r >> top) & 1 else r for r in rows]
    return rank


@pytest.mark.parametrize("key", sorted(CODES))
def test_code_parameters(key):
    n, k, d = CODES[key]
    code = C.code_by_name(key)
    assert code.n == n
    hx, hz = code.hx.astype(np.int64), code.hz.astype(np.int64)
    assert not ((hx @ hz.T) % 2).any()
    assert n - gf2_rank_plain(hx) - gf2_rank_plain(hz) == k
    if key.startswith("bb"):
        assert (hx.sum(1) == 6).all() and (hz.sum(1) == 6).all()
    # logical Z operators commute with X checks, are independent modulo Z checks
    zl = np.zeros((len(code.z_logicals), n), dtype=np.int64)
    for i, s in enumerate(code.z_logicals):
        zl[i, s] = 1
    assert len(code.z_logicals) == k
    assert not ((hx @ zl.T) % 2).any()
    assert gf2_rank_plain(np.vstack([hz, zl])) == gf2_rank_plain(hz) + k
    if key.startswith("sc"):
        assert all(len(s) == d for s in code.z_logicals)


@pytest.mark.parametrize("key", sorted(T3))
def test_table_iii_counts(key):
    exp = T3[key]
    code = C.code_by_name(key)
    nl = C.gate_counts(C.nonlocal_cnot_circuit(code, 4, 3))
    tp = C.gate_counts(C.teleport_circuit(code, 4, 3))
    assert [nl["1q"], nl["2q"], nl["M"], nl["rows"]] == exp[0:4]
    assert [tp["1q"], tp["2q"], tp["M"], tp["rows"]] == exp[5:9]


@pytest.mark.parametrize("key", ["sc3", "sc5"])
def test_table_iii_dem_columns_surface(key):
    """DEM column counts of the surface-code circuits equal Table III."""
    from oracle import dem
    exp = T3[key]
    code = C.code_by_name(key)
    assert len(dem.columns(C.nonlocal_cnot_circuit(code, 4, 3))) == exp[4]
    assert len(dem.columns(C.teleport_circuit(code, 4, 3))) == exp[9]


def test_table_iii_dem_columns_bb_nonlocal():
    """BB non-local CNOT columns match Table III for [[18,4,4]] (soft pin:
    the BB syndrome schedule is this project's own)."""
    from oracle import dem
    code = C.code_by_name("bb18")
    assert len(dem.columns(C.nonlocal_cnot_circuit(code, 4, 3))) == T3["bb18"][4]


@pytest.mark.parametrize("key", ["sc3", "sc5", "bb18", "bb36"])
@pytest.mark.parametrize("kind", ["memory", "nl", "teleport"])
def test_detectors_deterministic(key, kind):
    import oracle
    code = C.code_by_name(key)
    if kind == "memory":
        c = C.memory_circuit(code, 3)
    elif kind == "nl":
        c = C.nonlocal_cnot_circuit(code, 2, 2)
    else:
        c = C.teleport_circuit(code, 2, 2)
    bad_d, bad_o = oracle.gauge_audit(c)
    assert bad_d.size == 0 and bad_o.size == 0


def test_workload_sizes():
    """Sizes of the named workloads (detectors, observables, qubits)."""
    c = C.WORKLOADS["nl_sc3"].circuit()
    assert (c.n_qubits, c.n_det, c.n_obs) == (52, 56, 2)
    c = C.WORKLOADS["nl_sc11"].circuit()
    assert (c.n_qubits, c.n_det, c.n_obs, c.n_meas) == (724, 2760, 2, 5764)
    c = C.WORKLOADS["tp_bb144"].circuit()
    assert (c.n_qubits, c.n_det, c.n_obs) == (1152, 72 * (3 * 12 + 12 + 1), 12)


def test_text_roundtrip():
    c = C.teleport_circuit(C.code_by_name("sc3"), 1, 1)
    t = c.to_text()
    c2 = C.Circuit.from_text(t)
    assert c2.to_text() == t
    assert (c2.n_qubits, c2.n_meas, c2.n_det, c2.n_obs) == (c.n_qubits, c.n_meas, c.n_det, c.n_obs)


def test_invalid_ops_rejected():
    c = C.Circuit()
    with pytest.raises(ValueError):
        c.append("CX", [0, 1, 2])
    with pytest.raises(ValueError):
        c.append("X_ERROR", [0], p=1.5)
    with pytest.raises(ValueError):
        c.append("DETECTOR", [0])
    with pytest.raises(ValueError):
        c.append("FOO", [0])


@pytest.mark.parametrize("key", ["sc3", "bb18"])
@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 6])
def test_pauli_string_chain_deterministic(key, w):
    """Methods "Pauli string compute": w+1 blocks, the chain pattern of the
    text (w=2: 1, 3: 10, 4: 101, 5: 1010, 6: 10101), all detectors and
    observables deterministic, one ebit pair per data qubit per non-local link."""
    import oracle
    code = C.code_by_name(key)
    c = C.pauli_string_circuit(code, w, rounds_before=2, noise=C.NoiseModel(1e-3, 1e-3))
    bad_d, bad_o = oracle.gauge_audit(c)
    assert bad_d.size == 0 and bad_o.size == 0
    nonlocal_links = C.CHAIN_PATTERNS.get(w, "").count("1")
    # qubits: (w+1) blocks of data + check ancillas, plus 2n ebits per non-local link
    per_block = code.n + code.n_xchecks + code.n_zchecks
    assert c.n_qubits == (w + 1) * per_block + nonlocal_links * 2 * code.n
    assert c.n_obs == (w + 1) * code.k


def test_pauli_string_distance_sc3():
    """The chained compute on distance-3 surface-code blocks keeps circuit
    distance 3 (same check as Table I's for the paper's primitives)."""
    from oracle import dem
    c = C.pauli_string_circuit(C.code_by_name("sc3"), 3, rounds_before=2, noise=C.NoiseModel(1e-3, 1e-3))
    assert dem.circuit_distance(c, max_weight=3) == 3


def test_pauli_string_pattern_validation():
    with pytest.raises(ValueError):
        C.pauli_string_circuit(C.code_by_name("sc3"), 3, pattern="1")
    with pytest.raises(ValueError):
        C.pauli_string_circuit(C.code_by_name("sc3"), 3, pattern="12")


def test_decoherence_channel_limits():
    """Methods "Decoherence": no idling gives no noise; an ebit idle for many
    T1 = T2 is fully depolarised (X, Y, Z each 1/4); short idling costs
    t / (4 T1) per Pauli."""
    assert C.decoherence_paulis(0.0, 0.0) == (0.0, 0.0, 0.0)
    px, py, pz = C.decoherence_paulis(60.0, 60.0)
    assert abs(px - 0.25) < 1e-12 and abs(py - 0.25) < 1e-12 and abs(pz - 0.25) < 1e-12
    px, py, pz = C.decoherence_paulis(1e-6, 1e-6)
    assert abs(px / 2.5e-7 - 1) < 1e-5 and abs(pz / 2.5e-7 - 1) < 1e-5


@pytest.mark.parametrize("schedule", ["serial", "lines"])
def test_decoherence_ebit_ages(schedule):
    """Serial generation ages ebit j by (n - j) t_gen; line generation (f = d
    per step for the surface code) ages line l by (L - l) t_gen; every ebit
    half gets its channel and the circuit stays deterministic."""
    import oracle
    code = C.code_by_name("sc5")
    dec = C.Decoherence(1e-3, schedule=schedule)
    c = C.nonlocal_cnot_circuit(code, 2, 2, C.NoiseModel(1e-3, 1e-2, decoherence=dec))
    pcs = [op for op in c.ops if op.name == "PAULI_CHANNEL_1"]
    ages = sorted(round(-4 * __import__("math").log1p(-4 * op.channel[0]) / 1e-3 / 4) for op in pcs)
    if schedule == "serial":
        assert ages == list(range(1, 25)) and all(op.targets.size == 2 for op in pcs)
    else:
        assert ages == [1, 2, 3, 4] and all(op.targets.size == 10 for op in pcs)
    bad_d, bad_o = oracle.gauge_audit(c)
    assert bad_d.size == 0 and bad_o.size == 0


def test_line_width_bb():
    """BB codes use the divisor of n closest to d (Methods "Decoherence")."""
    assert C.line_width(C.code_by_name("bb144"), 144) == 12
    assert C.line_width(C.code_by_name("bb18"), 18) == 3
    assert C.line_width(C.code_by_name("bb90"), 90) == 10
