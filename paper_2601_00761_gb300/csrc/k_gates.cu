// k_gates.cu -- H, S, S^dag, T, T^dag, CNOT and general two-qubit gates
// (4x4 complex matrices) on a complex64 state vector (the Clifford
// preconditioning circuits, T doping and brick-wall circuits of the paper), applied
// in fused blocks: a run of consecutive gates acting inside a set of at most
// GATE_BLOCK_Q qubits (always containing qubits 0..4, so every tile is made of
// 256-byte contiguous runs) is applied to each 2^Q-amplitude tile in shared
// memory with one global read and one global write of psi per block.
#include "k_misc.cuh"

namespace sre {

struct GateBlockParams {
    int Q;                       // qubits in the block
    int n_other;                 // qubits outside the block
    unsigned char local[GATE_BLOCK_Q];   // global qubit of local bit i (ascending)
    unsigned char other[32];             // global qubit of tile bit i (ascending)
    int g0, ng;                  // gate rows [g0, g0 + ng) of the translated list
};

__global__ void __launch_bounds__(256) gate_block_kernel(float2 *psi, const GateRow *gates, const float2 *mats,
                                                         GateBlockParams p) {
    extern __shared__ __align__(16) float2 amp[];
    __shared__ unsigned long long hioff[1 << (GATE_BLOCK_Q - GATE_BLOCK_LOW)];
    const unsigned long long tile = blockIdx.x + ((unsigned long long)blockIdx.y << 15);
    if (tile >= (1ULL << p.n_other)) return;   // uniform over the CTA
    unsigned long long base = 0;
    for (int i = 0; i < p.n_other; ++i) base |= ((tile >> i) & 1ULL) << p.other[i];
    const int L = 1 << p.Q;
    // local bits 0..LOW-1 are global bits 0..LOW-1 (contiguous runs); the
    // global offset of the remaining local bits h = l >> LOW, one table entry
    // per value of h
    const int low = p.Q < GATE_BLOCK_LOW ? p.Q : GATE_BLOCK_LOW;
    const int nh = 1 << (p.Q - low);
    for (int h = threadIdx.x; h < nh; h += 256) {
        unsigned long long o = base;
        for (int i = low; i < p.Q; ++i) o |= (unsigned long long)((h >> (i - low)) & 1) << p.local[i];
        hioff[h] = o;
    }
    // the block's two-qubit matrices, once per CTA (read back as broadcasts)
    float2 *msm = amp + L;
    if (mats)
        for (int e = threadIdx.x; e < 16 * p.ng; e += 256) msm[e] = __ldg(mats + 16 * (size_t)p.g0 + e);
    __syncthreads();
    const int lm = (1 << low) - 1;
    for (int l = threadIdx.x; l < L; l += 256) amp[l] = psi[hioff[l >> low] | (unsigned long long)(l & lm)];
    const float r2 = 0.70710678118654752440f;
    for (int gi = 0; gi < p.ng; ++gi) {
        const GateRow G = gates[p.g0 + gi];
        __syncthreads();
        const int b0 = 1 << G.q0;
        if (G.op == GATE_OP_U2) {   // 4x4 matrix of row p.g0 + gi, local index bit(q0) + 2 bit(q1)
            const float2 *u = msm + 16 * gi;
            float2 m[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) m[e] = u[e];
            const int b1 = 1 << G.q1;
            const int lo = G.q0 < G.q1 ? G.q0 : G.q1, hi = G.q0 < G.q1 ? G.q1 : G.q0;
            for (int pi = threadIdx.x; pi < L / 4; pi += 256) {
                int i = ((pi >> lo) << (lo + 1)) | (pi & ((1 << lo) - 1));
                i = ((i >> hi) << (hi + 1)) | (i & ((1 << hi) - 1));
                const int idx[4] = {i, i | b0, i | b1, i | b0 | b1};
                float2 v[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) v[l] = amp[idx[l]];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float re = 0.f, im = 0.f;
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        re = fmaf(m[4 * r + l].x, v[l].x, fmaf(-m[4 * r + l].y, v[l].y, re));
                        im = fmaf(m[4 * r + l].x, v[l].y, fmaf(m[4 * r + l].y, v[l].x, im));
                    }
                    amp[idx[r]] = make_float2(re, im);
                }
            }
        } else if (G.op == 0) {   // H
            for (int pi = threadIdx.x; pi < L / 2; pi += 256) {
                const int i = ((pi >> G.q0) << (G.q0 + 1)) | (pi & (b0 - 1));
                const float2 u = amp[i], w = amp[i | b0];
                amp[i] = make_float2(r2 * (u.x + w.x), r2 * (u.y + w.y));
                amp[i | b0] = make_float2(r2 * (u.x - w.x), r2 * (u.y - w.y));
            }
        } else if (G.op == 3) {   // CNOT q0 -> q1
            const int b1 = 1 << G.q1;
            const int lo = G.q0 < G.q1 ? G.q0 : G.q1, hi = G.q0 < G.q1 ? G.q1 : G.q0;
            for (int pi = threadIdx.x; pi < L / 4; pi += 256) {
                int i = ((pi >> lo) << (lo + 1)) | (pi & ((1 << lo) - 1));
                i = ((i >> hi) << (hi + 1)) | (i & ((1 << hi) - 1));
                i |= b0;
                const float2 u = amp[i];
                amp[i] = amp[i | b1];
                amp[i | b1] = u;
            }
        } else {   // diagonal phase on |1> of q0
            float cr, ci;
            if (G.op == 1) { cr = 0.f; ci = 1.f; }
            else if (G.op == 2) { cr = 0.f; ci = -1.f; }
            else if (G.op == 4) { cr = r2; ci = r2; }
            else { cr = r2; ci = -r2; }
            for (int pi = threadIdx.x; pi < L / 2; pi += 256) {
                const int i = ((pi >> G.q0) << (G.q0 + 1)) | (pi & (b0 - 1)) | b0;
                const float2 u = amp[i];
                amp[i] = make_float2(cr * u.x - ci * u.y, cr * u.y + ci * u.x);
            }
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += 256) psi[hioff[l >> low] | (unsigned long long)(l & lm)] = amp[l];
}

// blocks_host: n_blocks x (g0, ng); block_qubits_host: n_blocks x GATE_BLOCK_Q
// global qubits (ascending, 255 = unused). Gate rows in gates_dev carry local
// qubit positions.
cudaError_t launch_gate_blocks(float2 *psi, int N, const GateRow *gates_dev, const float2 *mats_dev,
                               const int *blocks_host, int n_blocks, const unsigned char *block_qubits_host,
                               cudaStream_t st) {
    int max_ng = 0;
    for (int b = 0; b < n_blocks; ++b) max_ng = blocks_host[2 * b + 1] > max_ng ? blocks_host[2 * b + 1] : max_ng;
    const size_t mat_smem = mats_dev ? sizeof(float2) * 16 * (size_t)max_ng : 0;
    const size_t smem_max = (sizeof(float2) << GATE_BLOCK_Q) + mat_smem;
    if (smem_max > 200 * 1024) return cudaErrorInvalidValue;
    static size_t attr = 0;
    if (attr < smem_max) {
        cudaError_t e = cudaFuncSetAttribute(gate_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_max);
        if (e != cudaSuccess) return e;
        attr = smem_max;
    }
    for (int b = 0; b < n_blocks; ++b) {
        GateBlockParams p;
        p.g0 = blocks_host[2 * b];
        p.ng = blocks_host[2 * b + 1];
        p.Q = 0;
        bool in[64] = {false};
        for (int i = 0; i < GATE_BLOCK_Q; ++i) {
            const unsigned char q = block_qubits_host[b * GATE_BLOCK_Q + i];
            if (q == 255) break;
            p.local[p.Q++] = q;
            in[q] = true;
        }
        p.n_other = 0;
        for (int q = 0; q < N; ++q)
            if (!in[q]) p.other[p.n_other++] = (unsigned char)q;
        const unsigned long long tiles = 1ULL << p.n_other;
        dim3 grid((unsigned)(tiles < 32768 ? tiles : 32768), (unsigned)(tiles < 32768 ? 1 : tiles >> 15));
        const size_t smem = (sizeof(float2) << p.Q) + (mats_dev ? sizeof(float2) * 16 * (size_t)p.ng : 0);
        gate_block_kernel<<<grid, 256, smem, st>>>(psi, gates_dev, mats_dev, p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace sre
