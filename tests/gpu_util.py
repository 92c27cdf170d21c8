"""Helpers shared by the GPU tests: device copies of string sets and the
edge-case sets used for parity."""
import numpy as np

import synth


def to_device(s, device="cuda:0"):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(s.bytes)).to(device),
            torch.from_numpy(np.ascontiguousarray(s.offsets)).to(device))


def edge_set(seed: int = 0) -> synth.StringSet:
    """Empty strings (first, middle, last), strings shorter than q, single
    symbols, periodic runs, long strings spanning several 4096-byte tiles,
    and near-duplicate families: the degenerate cases of Alg. 1-3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = synth.DNA
    strs = [b""]
    for L in (1, 2, 3, 5, 8, 9, 10, 11, 17):
        strs.append(A[rng.integers(0, 4, size=L)].tobytes())
    strs += [b"", b"A" * 50, b"AC" * 40, b"ACG" * 30, b"A" * 9000]
    root = A[rng.integers(0, 4, size=9000)]
    for _ in range(4):
        strs.append(synth.mutate(rng, root, 0.003, A).tobytes())
    root2 = A[rng.integers(0, 4, size=300)]
    for _ in range(6):
        strs.append(synth.mutate(rng, root2, 0.01, A).tobytes())
    for _ in range(40):
        strs.append(A[rng.integers(0, 4, size=int(rng.integers(20, 400)))].tobytes())
    strs.append(root2.tobytes())
    strs.append(b"")
    return synth.from_strings(strs, K=8, T=8, name="edge cases")


def parity_sets():
    """(name, factory) of the string sets used for element-wise parity."""
    return [
        ("config1", lambda: synth.make_config(1)),
        ("config2_20roots", lambda: synth.make_config(2, n_roots=20)),
        ("config3_6roots", lambda: synth.make_config(3, n_roots=6)),
        ("config4_400roots", lambda: synth.make_config(4, n_roots=400)),
        ("config5_120roots", lambda: synth.make_config(5, n_roots=120)),
        ("edge", lambda: edge_set(0)),
        ("random_mixed", lambda: synth.random_set(5, n=300, min_len=1, max_len=700, K=6, T=6,
                                                  families=12, rate=0.02)),
    ]
