"""Seeded random test circuits (inputs only; no sampling arithmetic)."""
from paper_2504_05611_gb300 import circuits as C


def random_noisy_circuit(rng, n, depth):
    """Random Clifford body + inverse on |0>/|+> inputs with noise sprinkled
    in, a mid-circuit measurement feeding conditioned Paulis, and one detector
    per (deterministic) final measurement."""
    c = C.Circuit()
    xb = [q for q in range(n) if rng.random() < 0.4]
    zb = [q for q in range(n) if q not in xb]
    if zb:
        c.append("R", zb)
    if xb:
        c.append("RX", xb)
    body = []
    for _ in range(depth):
        u = rng.integers(3)
        if u == 0:
            body.append(("H", [int(rng.integers(n))]))
        elif u == 1:
            body.append(("S", [int(rng.integers(n))]))
        else:
            a, b = rng.choice(n, 2, replace=False)
            body.append(("CX", [int(a), int(b)]))
    inv = []
    for name, t in reversed(body):
        inv += [("S", t)] * 3 if name == "S" else [(name, t)]
    for i, (name, t) in enumerate(body + inv):
        c.append(name, t)
        if rng.random() < 0.3:
            kind = ["X_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2", "PAULI_CHANNEL_1"][int(rng.integers(5))]
            if kind == "PAULI_CHANNEL_1":
                qs = sorted(set(int(v) for v in rng.integers(0, n, 2)))
                c.append(kind, qs, p=tuple(float(v) for v in rng.uniform(0.0, 0.1, 3)))
            elif kind == "DEPOLARIZE2":
                a, b = rng.choice(n, 2, replace=False)
                c.append(kind, [int(a), int(b)], p=float(rng.uniform(0.01, 0.3)))
            else:
                qs = sorted(set(int(v) for v in rng.integers(0, n, 2)))
                c.append(kind, qs, p=float(rng.uniform(0.01, 0.3)))
    if zb:
        anc = n
        c.append("R", [anc])
        c.append("CX", [zb[0], anc])
        r = c.append("M", [anc])
        c.append("XFEED", [int(r[0]), int(rng.integers(n))])
        c.append("ZFEED", [int(r[0]), int(rng.integers(n))])
    if zb:
        c.append("M", zb)
    if xb:
        c.append("MX", xb)
    for r in range(c.n_meas):
        c.append("DETECTOR", [r])
    c.append("OBSERVABLE", [c.n_meas - 1], arg=0)
    return c
