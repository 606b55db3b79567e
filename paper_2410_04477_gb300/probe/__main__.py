import ctypes
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fp_peaks.cu")
LIB = os.path.join(HERE, "_build", "libbvprobe.so")


def build():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", "-o", LIB, SRC], check=True)
    return LIB


def main():
    lib = ctypes.CDLL(build())
    lib.bvp_fma_rate.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_double)]
    out = {}
    r = ctypes.c_double(0)
    for name, typ, iters in (("fp64", 0, 2048), ("fp32", 1, 16384)):
        for lanes in (32, 1):
            st = lib.bvp_fma_rate(typ, lanes, 152 * 8, 256, iters, ctypes.byref(r))
            out[f"{name}_lanes{lanes}_tflops"] = None if st else 2 * r.value / 1e12
    print(json.dumps(out))


if __name__ == "__main__":
    main()
