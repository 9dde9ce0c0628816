"""The library's modular arithmetic header, compiled for the host, agrees
with 128-bit integer '%' within its documented preconditions, for primes of
20..58 bits and the key inner product's largest admitted digit sums."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_modarith_against_int128(tmp_path):
    exe = str(tmp_path / "modarith_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "modarith_check.cpp")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
