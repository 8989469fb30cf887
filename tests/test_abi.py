"""C ABI checks that need no GPU: the library loads and exports every
function include/tmcs.h declares; host-side calls (compile, info, stats,
reference sample, gap tables) behave; invalid inputs are rejected with the
documented status codes."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_2504_05611_gb300 import build as lib_build
from paper_2504_05611_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tmcs():
    lib_build.build()
    from paper_2504_05611_gb300 import tmcs as t
    return t


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(tmcs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(tmcs):
    names = declared_functions()
    assert "tmcs_sample" in names and "tmcs_batch_sample" in names
    L = tmcs.lib()
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("p", [1e-4, 1e-3, 1e-2, 0.25, 1.0])
def test_gap_table_equals_oracle(tmcs, p):
    assert np.array_equal(tmcs.tmcs_debug_gap_table(p), oracle.gap_table(p))


@pytest.mark.parametrize("name", ["sc3", "bb18"])
@pytest.mark.parametrize("kind", ["nl", "teleport"])
def test_reference_sample_equals_oracle_tableau(tmcs, name, kind):
    code = C.code_by_name(name)
    fn = C.nonlocal_cnot_circuit if kind == "nl" else C.teleport_circuit
    c = fn(code, 2, 2)
    h = tmcs.tmcs_circuit_build(c)
    try:
        assert np.array_equal(tmcs.tmcs_reference_sample(h), tableau.reference_sample(c)["rec"])
    finally:
        tmcs.tmcs_circuit_free(h)


def test_info_and_pruning_stats(tmcs):
    c = C.WORKLOADS["nl_sc3"].circuit()
    h = tmcs.tmcs_circuit_build(c)
    info = tmcs.tmcs_circuit_info(h)
    assert (info["n_qubits"], info["n_meas"], info["n_det"], info["n_obs"]) == (52, 132, 56, 2)
    st = tmcs.tmcs_circuit_stats(h)
    # the non-local CNOT with Z detectors needs no z-plane: every z update pruned
    assert st["pruned_updates"] > 0 and st["n_slots"] > 0
    tmcs.tmcs_circuit_free(h)
    h = tmcs.tmcs_circuit_build(c, tmcs.TMCS_FLAG_NO_PRUNE)
    assert tmcs.tmcs_circuit_stats(h)["pruned_updates"] == 0
    tmcs.tmcs_circuit_free(h)


def test_rejects_nondeterministic_detector(tmcs):
    c = C.Circuit()
    c.append("RX", [0])
    c.append("M", [0])
    c.append("DETECTOR", [0])
    with pytest.raises(tmcs.TmcsError) as e:
        tmcs.tmcs_circuit_build(c)
    assert e.value.code == 2
    h = tmcs.tmcs_circuit_build(c, tmcs.TMCS_FLAG_NO_AUDIT)
    tmcs.tmcs_circuit_free(h)


def test_sample_rejects_bad_arguments_before_device_work(tmcs):
    """Argument errors come back before any device call, so these run
    without a GPU: misaligned or missing output buffers (TMCS_E_BUFFER = 6,
    TMCS_E_INVALID = 1), zero shots, a chunk range past 2^32, a NULL circuit
    or job list."""
    h = tmcs.tmcs_circuit_build(C.WORKLOADS["nl_sc3"].circuit())
    L = tmcs.lib()
    try:
        assert L.tmcs_sample(h, 64, 1, 0x1001, 0x2000, None) == 6
        assert "aligned" in tmcs.tmcs_last_error()
        assert L.tmcs_sample(h, 64, 1, 0x1000, 0x2004, None) == 6
        assert L.tmcs_sample(h, 0, 1, 0x1000, 0x2000, None) == 1
        assert L.tmcs_sample(h, 64, 1, None, 0x2000, None) == 1
        assert L.tmcs_sample(h, 64, 1, 0x1000, None, None) == 1
        assert L.tmcs_sample_range(h, (1 << 32) - 1, 128, 1, 0x1000, 0x2000, None) == 1
        # first chunks near 2^64 must not wrap the range check around
        for fc in ((1 << 64) - 1, (1 << 64) - 2, 1 << 32):
            assert L.tmcs_sample_range(h, fc, 128, 1, 0x1000, 0x2000, None) == 1
            assert L.tmcs_sample_noalloc(h, fc, 128, 1, 0x1000, 0x2000, None) == 1
            assert L.tmcs_sample_measurements(h, fc, 128, 1, 0x1000, None) == 1
            assert "2^32" in tmcs.tmcs_last_error()
        assert L.tmcs_sample(None, 64, 1, 0x1000, 0x2000, None) == 1
        assert L.tmcs_batch_sample(None, 3, None) == 1
    finally:
        tmcs.tmcs_circuit_free(h)


def test_rejects_invalid_ops(tmcs):
    arr = np.zeros(1, dtype=tmcs.OP_DTYPE)
    arr["code"] = 99
    import ctypes
    out = ctypes.c_void_p()
    assert tmcs.lib().tmcs_circuit_build(arr.ctypes.data, 1, 0, ctypes.byref(out)) == 1
    assert "opcode" in tmcs.tmcs_last_error()
    c = C.Circuit()
    c.append("X_ERROR", [0, 0], p=0.1)   # noise ops must hit distinct qubits
    with pytest.raises(tmcs.TmcsError):
        tmcs.tmcs_circuit_build(c)
    c = C.Circuit()
    c.append("X_ERROR", [0], p=1e-13)
    with pytest.raises(tmcs.TmcsError):
        tmcs.tmcs_circuit_build(c)
    with pytest.raises(tmcs.TmcsError):
        tmcs.tmcs_circuit_build(C.Circuit(), flags=0x80)
    # arg2 is only meaningful for PAULI_CHANNEL_1, whose thresholds must be ordered
    c = C.Circuit()
    c.append("R", [0])
    arr, flat = tmcs.marshal_ops(c)
    arr["arg2"] = 5
    assert tmcs.lib().tmcs_circuit_build(arr.ctypes.data, 1, 0, ctypes.byref(out)) == 1
    c = C.Circuit()
    c.append("PAULI_CHANNEL_1", [0], p=(0.1, 0.1, 0.1))
    arr, flat = tmcs.marshal_ops(c)
    arr["arg"], arr["arg2"] = arr["arg2"][0], arr["arg"][0]
    assert tmcs.lib().tmcs_circuit_build(arr.ctypes.data, 1, 0, ctypes.byref(out)) == 1


@pytest.mark.parametrize("trial", range(40))
def test_random_circuits_compile_and_validate(tmcs, trial):
    """The compiler's output passes its own program check (slot, block and
    window bounds the kernel relies on) for random circuits, pruned or not."""
    from circuit_gen import random_noisy_circuit
    rng = np.random.default_rng(300 + trial)
    c = random_noisy_circuit(rng, int(rng.integers(2, 12)), int(rng.integers(4, 80)))
    for flags in (0, tmcs.TMCS_FLAG_NO_PRUNE):
        h = tmcs.tmcs_circuit_build(c, flags)
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("kind", ["nl", "teleport"])
def test_fault_count_matches_oracle_enumeration(tmcs, kind):
    """The library's single-fault enumeration has the oracle DEM's length."""
    from oracle import dem
    nz = C.NoiseModel(1e-3, 1e-2, decoherence=C.Decoherence(1e-3, schedule="lines"))
    fn = C.nonlocal_cnot_circuit if kind == "nl" else C.teleport_circuit
    c = fn(C.code_by_name("sc3"), 2, 2, nz)
    h = tmcs.tmcs_circuit_build(c)
    try:
        assert tmcs.tmcs_fault_count(h) == len(dem.fault_list(c))
    finally:
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("kind", ["nl_sc5", "tp_bb18", "ps4_sc3", "random"])
def test_measurement_program_compiles_and_validates(tmcs, kind):
    """tmcs_sample_measurements builds its gauge/record program on the host
    (reference tableau, compile, program check) before any CUDA call; without
    a GPU it must then stop at the first CUDA call, not in the program check."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    if kind == "nl_sc5":
        c = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 2, 2, C.NoiseModel(0.001, 0.01))
    elif kind == "tp_bb18":
        c = C.teleport_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.001, 0.01))
    elif kind == "ps4_sc3":
        c = C.pauli_string_circuit(C.code_by_name("sc3"), 4, rounds_before=1, noise=C.NoiseModel(0.003, 0.02))
    else:
        from circuit_gen import random_noisy_circuit
        c = random_noisy_circuit(np.random.default_rng(5), 6, 30)
    h = tmcs.tmcs_circuit_build(c)
    try:
        rc = tmcs.lib().tmcs_sample_measurements(h, 0, 64, 1, 4096, None)
        assert rc == 4, tmcs.tmcs_last_error()
        assert "program check" not in tmcs.tmcs_last_error()
    finally:
        tmcs.tmcs_circuit_free(h)


def _sig_cases():
    from circuit_gen import random_noisy_circuit
    out = [("nl_sc3", C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.05))),
           ("tp_sc3", C.teleport_circuit(C.code_by_name("sc3"), 1, 1, C.NoiseModel(0.01, 0.05))),
           ("nl_bb18", C.nonlocal_cnot_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.01, 0.05))),
           ("ps3_sc3", C.pauli_string_circuit(C.code_by_name("sc3"), 3, rounds_before=1,
                                              noise=C.NoiseModel(0.01, 0.01))),
           ("deco_sc3", C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 1, 1,
                                                C.NoiseModel(0.003, 0.02, decoherence=C.Decoherence(0.05))))]
    for t in range(6):
        rng = np.random.default_rng(1700 + t)
        out.append((f"rand{t}", random_noisy_circuit(rng, int(rng.integers(2, 9)), int(rng.integers(4, 40)))))
    return out


@pytest.mark.parametrize("case", _sig_cases(), ids=lambda c: c[0])
def test_event_signatures_equal_oracle_dem(tmcs, case):
    """The host event-signature table (transposed frame pass) gives, for every
    elementary fault, exactly the detectors and observables the oracle's
    forward single-fault propagation flips."""
    from oracle import dem
    _, circ = case
    dets, obss, _, _ = dem.signatures(circ)
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == 1
        assert tmcs.tmcs_fault_count(h) == len(dets)
        for f, (dm, om) in enumerate(zip(dets, obss)):
            gd, go = tmcs.tmcs_fault_outputs(h, f)
            assert gd == [j for j in range(circ.n_det) if dm >> j & 1], f
            assert go == [j for j in range(circ.n_obs) if om >> j & 1], f
    finally:
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("window", [1024, 2048])
def test_signature_window_forces_steps(tmcs, window, monkeypatch):
    """A detector ring smaller than the circuit's detector count splits the
    noise segments into several flush steps; every segment is walked."""
    monkeypatch.setenv("TMCS_SIG_WINDOW", str(window))
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.001, 0.01))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        st = tmcs.tmcs_circuit_stats(h)
        assert st["sig_ok"] == 1 and st["sig_window"] == window and st["sig_steps"] > 1
        assert st["sig_items"] == st["n_noise_segments"]
    finally:
        tmcs.tmcs_circuit_free(h)


def test_signature_schedules_halve_the_ring(tmcs):
    """The program carries up to three schedules whose rings halve from the
    main one down to the smallest feasible power of two (>= 1024); a
    1024-detector main ring leaves a single schedule."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.001, 0.01))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        st = tmcs.tmcs_circuit_stats(h)
        assert st["sig_ok"] == 1 and st["sig_window"] == 4096
        assert st["sig_schedules"] == 3 and st["sig_min_window"] == 1024
    finally:
        tmcs.tmcs_circuit_free(h)


def test_signature_single_schedule_at_the_floor(tmcs, monkeypatch):
    monkeypatch.setenv("TMCS_SIG_WINDOW", "1024")
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.001, 0.01))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        st = tmcs.tmcs_circuit_stats(h)
        assert st["sig_schedules"] == 1 and st["sig_min_window"] == st["sig_window"] == 1024
    finally:
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("mistake,reason", [("observable", "event entry"), ("record", "item record"),
                                            ("window", "window"), ("live", "walker descriptor")])
def test_signature_validator_refuses_planted_mistakes(tmcs, monkeypatch, mistake, reason):
    """The host-side validator of the event-signature program refuses a
    program with an out-of-range observable id, a wrong item record, a ring
    too small for its steps, or a walker descriptor whose live-Pauli mask
    leaves out a Pauli index that flips an output (the decoupled kernel would
    drop those events); the circuit then has no signature program (sampling
    runs on the frame kernels)."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.001, 0.01))
    h = tmcs.tmcs_circuit_build(circ)
    assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == 1
    tmcs.tmcs_circuit_free(h)
    monkeypatch.setenv("TMCS_TEST_CORRUPT_SIG", mistake)
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == 0
        with pytest.raises(tmcs.TmcsError) as err:
            tmcs.tmcs_fault_outputs(h, 0)
        assert "internal" in str(err.value) and reason in str(err.value)
    finally:
        tmcs.tmcs_circuit_free(h)


def _long_span_circuit(n_mid):
    """An X error on qubit 0 flips detector 0 (first measurement) and the last
    detector (second measurement, after n_mid other detectors)."""
    c = C.Circuit()
    c.append("R", [0])
    c.append("X_ERROR", [0], p=0.1)
    r0 = c.append("M", [0])
    c.append("DETECTOR", [int(r0[0])])
    c.append("R", list(range(1, n_mid + 1)))
    c.append("X_ERROR", list(range(1, n_mid + 1)), p=0.01)
    rs = c.append("M", list(range(1, n_mid + 1)))
    for r in rs:
        c.append("DETECTOR", [int(r)])
    r1 = c.append("M", [0])
    c.append("DETECTOR", [int(r1[0])])
    c.append("OBSERVABLE", [int(r1[0])], arg=0)
    return c


def test_signature_program_refuses_spans_beyond_the_ring(tmcs, monkeypatch):
    """A fault whose detectors lie further apart than the ring allows makes
    the event-signature program unusable (sampling then uses the frame
    kernels); a larger ring accepts the same circuit."""
    circ = _long_span_circuit(1500)
    monkeypatch.setenv("TMCS_SIG_WINDOW", "1024")
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == 0
    finally:
        tmcs.tmcs_circuit_free(h)
    monkeypatch.setenv("TMCS_SIG_WINDOW", "2048")
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == 1
    finally:
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("case", _sig_cases(), ids=lambda c: c[0])
def test_dem_columns_equal_oracle(tmcs, case):
    """tmcs_dem_columns (the parity-check-matrix columns of Methods
    "Decoding") equals the oracle's single-fault DEM merged by signature:
    the same columns, each with the oracle's odd-parity probability and fault
    count, in ascending order of their entry lists."""
    from oracle import dem
    _, circ = case
    want = dem.column_probabilities(circ)
    h = tmcs.tmcs_circuit_build(circ)
    try:
        cols, p, nf = tmcs.tmcs_dem_columns(h)
    finally:
        tmcs.tmcs_circuit_free(h)
    keys = [(sum(1 << j for j in d), sum(1 << j for j in o)) for d, o in cols]
    assert len(set(keys)) == len(keys) and set(keys) == set(want)
    for k, pc, n in zip(keys, p, nf):
        assert n == want[k][1]
        assert abs(pc - want[k][0]) <= 1e-12 + 1e-9 * want[k][0]
    entries = [d + [0x80000000 | o for o in ob] for d, ob in cols]
    assert entries == sorted(entries)


@pytest.mark.parametrize("key", ["sc3", "sc5", "sc7", "sc9", "sc11"])
def test_dem_columns_reproduce_table_iii(tmcs, key):
    """Distinct single-fault signatures of the 4/3-round surface-code
    circuits equal the "cols" of Table III (non-local CNOT and teleportation),
    computed by the library's C call."""
    from conftest import golden_rows
    t3 = {r[0]: [int(v) for v in r[1:]] for r in golden_rows("table_iii_counts.txt")}
    code = C.code_by_name(key)
    for fn, idx in ((C.nonlocal_cnot_circuit, 4), (C.teleport_circuit, 9)):
        h = tmcs.tmcs_circuit_build(fn(code, 4, 3))
        try:
            cols, _, _ = tmcs.tmcs_dem_columns(h)
            assert len(cols) == t3[key][idx]
        finally:
            tmcs.tmcs_circuit_free(h)


def test_dem_columns_buffer_contract(tmcs):
    """Sizes first, then arrays; too-small capacities return TMCS_E_BUFFER."""
    import ctypes
    h = tmcs.tmcs_circuit_build(C.WORKLOADS["nl_sc3"].circuit())
    L = tmcs.lib()
    try:
        nc, ne = ctypes.c_uint64(0), ctypes.c_uint64(0)
        assert L.tmcs_dem_columns(h, ctypes.byref(nc), ctypes.byref(ne), None, None, None, None) == 0
        assert nc.value > 0 and ne.value >= nc.value
        off = np.zeros(nc.value + 1, dtype=np.uint64)
        small = ctypes.c_uint64(nc.value - 1)
        assert L.tmcs_dem_columns(h, ctypes.byref(small), ctypes.byref(ne), off.ctypes.data, None, None, None) == 6
        assert L.tmcs_dem_columns(None, ctypes.byref(nc), ctypes.byref(ne), None, None, None, None) == 1
    finally:
        tmcs.tmcs_circuit_free(h)
