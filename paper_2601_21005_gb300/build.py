"""Build libsgw.so (the CUDA sm_103a library behind include/sgw.h) in-tree.

    python -m paper_2601_21005_gb300.build [--verbose]

Each translation unit is compiled by nvcc in parallel for sm_103a only, then linked
into paper_2601_21005_gb300/_build/libsgw.so (static CUDA runtime).
"""
import os
import subprocess
import sys
import concurrent.futures as cf

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, '_build')
LIB = os.path.join(OUT, 'libsgw.so')
SOURCES = ['kernels_grid.cu', 'kernels_rows.cu', 'kernels_cluster.cu', 'kernels_lines288.cu', 'kernels_misc.cu',
           'kernels_mlp.cu', 'abi.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '--expt-relaxed-constexpr']


def nvcc():
    for c in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return 'nvcc'


def _stale(objs):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, '..', 'include', 'sgw.h'), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose=False, ptxas_info=False, force=False):
    os.makedirs(OUT, exist_ok=True)
    objs = [os.path.join(OUT, s.replace('.cu', '.o')) for s in SOURCES]
    if not force and not _stale(objs):
        return LIB
    extra = ['-Xptxas', '-v'] if ptxas_info else []

    def comp(src, obj):
        cmd = [nvcc()] + ARCH + FLAGS + extra + ['-c', os.path.join(CSRC, src), '-o', obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda so: comp(*so), zip(SOURCES, objs)))
    for cmd, r in results:
        if verbose or ptxas_info or r.returncode != 0:
            sys.stderr.write(' '.join(cmd) + '\n' + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError('nvcc failed for ' + cmd[-3])
    tmp = LIB + '.tmp'
    cmd = [nvcc()] + ARCH + ['-shared', '-o', tmp] + objs + ['-lcudart_static', '-lrt', '-ldl', '-lpthread']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(' '.join(cmd) + '\n' + r.stdout + r.stderr)
        raise RuntimeError('link failed')
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    build(verbose='--verbose' in sys.argv, ptxas_info='--ptxas' in sys.argv, force=True)
    print(LIB)
