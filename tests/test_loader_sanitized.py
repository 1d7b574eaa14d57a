"""The loader's host code (decoder, validator, pruning, code generator), the
PREX check and plan, the input mutator, and the CPU oracle, each built with AddressSanitizer
and UndefinedBehaviorSanitizer and run over every workload program and
random PREX-shaped programs, each as given and with random byte mutations
(most rejected by the validators, some valid but unusual), with inputs at
the launch and argument extremes.  Any out-of-bounds access, leak, overflow
of a signed integer or other undefined behaviour fails the test."""
import os
import shutil
import struct
import subprocess

import pytest

from paper_2601_01048_gb300 import build_ext, gen

CSRC = os.path.join(os.path.dirname(build_ext.__file__), "csrc")
HERE = os.path.dirname(os.path.abspath(__file__))
EXTREMES = [0, 1, -1, 2**31 - 1, -2**31, 2**30, -2**30, 7, 1024, 65535]


SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]


def compile_or_skip(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "asan" in (r.stderr + r.stdout).lower():
        pytest.skip("sanitizer runtime not available")
    assert r.returncode == 0, r.stderr[-4000:]


def build_loader_driver(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    try:
        cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build_ext.nvcc())), "include")
    except RuntimeError:
        pytest.skip("no CUDA toolkit headers")
    exe = str(tmp_path / "loader_sanitized")
    compile_or_skip([gxx, "-std=c++17", *SAN, "-I", cuda_inc, "-I", CSRC,
                     "-x", "c++", os.path.join(CSRC, "loader.cpp"), os.path.join(CSRC, "prex.cpp"),
                     os.path.join(CSRC, "mutate.cpp"),
                     os.path.join(HERE, "sanitize", "loader_driver.cpp"), "-o", exe])
    return exe


def build_oracle_driver(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    exe = str(tmp_path / "oracle_sanitized")
    compile_or_skip([gcc, "-std=c11", *SAN, os.path.join(HERE, "sanitize", "oracle_driver.c"),
                     "-o", exe])
    return exe


def corpus(path, seed=0x5A17, mutations=10):
    from test_oracle_pins import affine_program
    from test_prex import affine_with_extras, guarded_1d_program
    rng = gen.SplitMix64(seed)
    progs = ([gen.c1_program()] + gen.c2_programs() + gen.c3_programs() + gen.c4_programs()
             + gen.affine_programs() + gen.c5_programs()[:8] + gen.div_programs()
             + gen.heap_programs() + gen.barrier_programs(8)
             + gen.barrier_programs(8, live=True))
    for _ in range(20):
        progs += [guarded_1d_program(rng), affine_with_extras(rng, 1 + rng.below(3)),
                  affine_program(rng, 1 + rng.below(3), 4)]

    def inputs(k):
        x = gen.make_inputs(k)
        for i in range(k):
            dims = rng.below(4)
            if dims == 0:
                grid = [rng.choice([0, 1, 2, 65535, 65536, 2**31 - 1]) for _ in range(3)]
                block = [rng.choice([0, 1, 32, 1024, 1025]) for _ in range(3)]
            else:
                grid = [rng.randint(1, 70) if d < dims else 1 for d in range(3)]
                block = [rng.randint(1, 64) if d < dims else 1 for d in range(3)]
            args = [rng.choice(EXTREMES) if rng.below(2) else rng.randint(-100, 100) for _ in range(4)]
            lens = [rng.choice([0, 1, 3, 4, 100, 4096, 2**40, 2**47]) for _ in range(9)]
            gen.set_input(x[i], 0, tuple(grid), tuple(block), tuple(args), tuple(lens))
        return x

    n = 0
    with open(path, "wb") as f:
        for p in progs:
            variants = [p]
            for _ in range(mutations):
                m = bytearray(p)
                for _ in range(1 + rng.below(4)):
                    j = rng.below(len(m))
                    m[j] = rng.below(256) if rng.below(2) else m[j] ^ (1 << rng.below(8))
                if rng.below(8) == 0:
                    m = m[: rng.below(len(m) + 1)]
                variants.append(bytes(m))
            for v in variants:
                x = inputs(4)
                f.write(struct.pack("<II", len(v), len(x)) + v + x.tobytes())
                n += 1
    return n


def run_clean(exe, path):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, path], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr[-4000:]
    return dict(zip(r.stdout.split()[0::2], map(int, r.stdout.split()[1::2])))


@pytest.fixture(scope="module")
def shared_corpus(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("corpus") / "corpus.bin")
    return path, corpus(path)


@pytest.fixture(scope="module")
def loader_counts(tmp_path_factory, shared_corpus):
    return run_clean(build_loader_driver(tmp_path_factory.mktemp("loader")), shared_corpus[0])


def test_loader_under_sanitizers(loader_counts, shared_corpus):
    assert loader_counts["programs"] == shared_corpus[1]
    assert loader_counts["valid"] > 150 and loader_counts["planned"] > 100


def test_oracle_under_sanitizers(tmp_path, shared_corpus, loader_counts):
    path, n = shared_corpus
    counts = run_clean(build_oracle_driver(tmp_path), path)
    assert counts["programs"] == n and counts["ran"] > 4 * 150
    # the two independent decoders accept the same programs
    assert counts["valid"] == loader_counts["valid"]
